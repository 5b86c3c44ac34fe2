/*
 * tac.h -- C ABI of the batched PNCG-IPC gel-pad contact solve.
 *
 * Each frame solves, for every pad of the batch, the implicit-Euler
 * incremental potential of the paper's Supplementary A, Eq. (ipc_energy):
 *
 *   E(x) = 1/2 (x - xhat)^T M (x - xhat) + h^2 Psi(x)
 *          + kappa * sum_{k in C} b(d_k(x)) + D(x),   xhat = x^t + h v^t,
 *
 * with Neo-Hookean Psi over linear tetrahedra, the C^2 log barrier b over
 * point-triangle / edge-edge pairs between the gel surface and a rigid
 * triangle-mesh indenter, and the lagged friction D of Eq. (friction_energy)
 * with the mollifier of Eq. (friction_mollifier). The minimiser is found by
 * the Dai-Kou preconditioned nonlinear CG of Eq. (dk_direction) with a 3x3
 * block-Jacobi preconditioner and the step rule of Eq. (step_size), bounded
 * by a per-pair conservative step (CCD) and accepted by an Armijo test.
 * Marker displacements are read out by barycentric interpolation of the
 * deformed mesh (Sec. 3.2, "Tactile Representation").
 *
 * Units are SI. A pad lives in its own frame: rest vertices in float32,
 * bottom-face Dirichlet vertices given explicitly, markers on the top face
 * (the face at maximum rest z). An indenter pose is a rotation vector (3)
 * followed by a translation (3) that maps the indenter's local vertices into
 * the pad frame.
 *
 * Conventions:
 *  - Every function returns TAC_OK (0) or a negative TAC_ERR_* code; the
 *    message of the last error on the calling thread is tac_last_error().
 *    The library never aborts and device code never traps: per-pad solve
 *    outcomes are TAC_PAD_* codes written to a caller-owned status array.
 *  - Host pointers (marked "host") are read during the call and may be freed
 *    afterwards. Device pointers (marked "device") belong to the caller and
 *    must stay valid until the stream-ordered work that reads or writes them
 *    has completed.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Every call is
 *    stream-ordered and asynchronous unless stated otherwise; results are
 *    visible after the stream is synchronised.
 *  - One device: the batch lives on the device that is current when
 *    tac_create_batch is called; later calls must be made with that device
 *    current.
 */
#ifndef TAC_H_
#define TAC_H_

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes --------------------------------------------------------- */
#define TAC_OK 0
#define TAC_ERR_INVALID_ARG (-1)   /* null / out-of-range argument               */
#define TAC_ERR_INVALID_MESH (-2)  /* bad index, non-positive tet volume, marker off the top face */
#define TAC_ERR_PENETRATION (-3)   /* gel and indenter intersect in the given state */
#define TAC_ERR_CUDA (-4)          /* a CUDA runtime call failed                 */
#define TAC_ERR_OOM (-5)           /* device allocation failed                   */
#define TAC_ERR_STATE (-6)         /* call not valid in the batch's current state */

/* ---- per-pad solve status (tac_step) -------------------------------------- */
#define TAC_PAD_CONVERGED 0        /* max |g_i| <= tol * g_ref at the end pose    */
#define TAC_PAD_MAXITER 1          /* max_iter PNCG iterations or 4000 indenter substeps in the frame */
#define TAC_PAD_NONFINITE 2        /* non-finite value met (state left as is)    */
#define TAC_PAD_LINESEARCH 3       /* 20 Armijo halvings without acceptance      */
#define TAC_PAD_PAIR_OVERFLOW 4    /* more contact candidates than pair_capacity */

typedef struct tac_batch* tac_handle;   /* opaque, library-owned */

/* One pad mesh (host arrays, copied at creation). */
typedef struct {
    int n_verts, n_tets, n_fixed, n_markers;
    const float* rest_xyz;   /* host [n_verts*3] rest positions                   */
    const int* tets;         /* host [n_tets*4] vertex ids, positive orientation */
    const int* fixed_idx;    /* host [n_fixed] Dirichlet vertex ids              */
    const float* marker_xy;  /* host [n_markers*2] marker (x, y) on the top face */
} tac_pad_desc;

/* One rigid indenter mesh per environment (host arrays, copied). */
typedef struct {
    int n_verts, n_tris;
    const float* verts;      /* host [n_verts*3] local frame                     */
    const int* tris;         /* host [n_tris*3]                                  */
} tac_indenter_desc;

/* Per-pad material and solver parameters.
 *  E, nu          Young's modulus [Pa] and Poisson ratio (Neo-Hookean Lame pair)
 *  rho, h         density [kg/m^3] and time step [s] (lumped mass; Eq. varopt)
 *  dhat           barrier activation distance [m] (Eq. ipc_energy)
 *  kappa          barrier stiffness; <= 0 selects h^2 * E * (mean surface edge)
 *  mu_f, eps_v    friction coefficient and mollifier width [m]; eps_v <= 0
 *                 selects 1e-3 m/s * h
 *  tol_rel_grad   stop when max |g_i| <= tol_rel_grad * g_ref with
 *                 g_ref = max(h^2 E (mean surface edge) dhat, max |g_i| at
 *                 the frame's first evaluation after the first indenter
 *                 substep); see tac_pad_norms for the float32 floor
 *  tol_advance    looser tolerance of the intermediate indenter substeps
 *  max_iter       PNCG iteration cap per frame
 *  precond_mode   0 = 3x3 block Jacobi, 1 = scalar Jacobi diag(H)^-1
 *                 (the literal preconditioner of Supp. A)
 *  step_mode      0 = alpha = min(alpha_upper, alpha_ccd, alpha_bar) with an
 *                 Armijo test (c = 1e-4, up to 20 halvings); 1 = Eq.
 *                 (step_size) as printed, alpha = min(alpha_upper, alpha_bar)
 *                 with no CCD bound and no energy test (a trial state that
 *                 inverts a tet or closes a gap is halved)
 *  marker_mode    0 = barycentric on the rest top-face triangle holding the
 *                 marker; 1 = the 4 rest top-face nodes nearest to the marker
 *                 (2-D distance, ties to the smaller id) with weights
 *                 proportional to 1/d (Sec. 3.2's kNN mapping). Fixed at
 *                 creation: tac_set_params rejects a change
 *  precision_mode 0 = the precision split of the solve: float32 elasticity
 *                 and CG vectors, double-float displacements, and float64
 *                 pair distance, barrier, step bounds and the sums that feed
 *                 the line search; 1 = the plain FP32 form of the same
 *                 method: single-float displacements and every distance,
 *                 barrier, bound and sum in float32 (the comparator the
 *                 split is measured against)
 *  floor_ulps     the float32 resolution floor of the stopping target in
 *                 ulps of the largest force component F summed into the
 *                 float32 gradient (elastic per-corner forces, barrier and
 *                 friction per-slot forces): the target is
 *                 max(tol_rel_grad * g_ref, floor_ulps * 2^-24 * F); <= 0
 *                 selects 256 (a float32 gradient is not resolved below a
 *                 few hundred ulps of the forces summed into it; a smaller
 *                 floor solves tighter where the line search can still
 *                 resolve the energy) */
typedef struct {
    float E, nu, rho, h, dhat, kappa, mu_f, eps_v;
    float tol_rel_grad, tol_advance;
    int max_iter, precond_mode, step_mode, marker_mode;
    int precision_mode;
    float floor_ulps;
} tac_params;

/* Batch options. pair_capacity: candidate pairs stored per pad (0 = 16384).
 * share_meshes: pads whose tac_pad_desc points at the same host arrays share
 * one device copy of the static mesh data (1) or each get their own (0).
 * no_dm_table: 0 (default) lets a mesh whose tets fall into at most 32
 * rest-shape classes (Dm^-1 equal within 1e-5 of their largest entry; a
 * regular hex-split grid has 6, one per tet of the cell split: the
 * structured-mesh case) read each tet's Dm^-1 from a per-mesh table of class
 * representatives instead of streaming one per tet; 1 always streams the
 * exact per-tet Dm^-1. The kernels form F = I + Du Dm^-1 from displacements,
 * so the table leaves the rest state exact and changes the strain of a
 * deformed tet by at most the class tolerance, relatively. */
typedef struct {
    int pair_capacity;
    int share_meshes;
    int no_dm_table;
} tac_options;

/* Create a batch of n_pads pads, pads_per_env consecutive pads per
 * environment (n_pads = n_envs * pads_per_env, at most 2^24), one indenter
 * per environment (Sec. 3.3: one sensor pad per finger of an environment,
 * each touched by the environment's object). The rest shape is what Eq.
 * (varopt) and Eq. (ipc_energy) are built on: per tet the inverse rest edge
 * matrix Dm^-1 and rest volume of the Neo-Hookean term, per vertex the
 * lumped mass rho V / 4 summed over its tets (the mass matrix M of the
 * inertia term), the gel surface whose vertices, triangles and edges form
 * the contact primitives of the set C, and the marker weights of Sec. 3.2. params has n_pads entries. opts may be NULL (defaults).
 * Validates every mesh on the host (TAC_ERR_INVALID_MESH with the pad index
 * in tac_last_error), builds the rest shape (Dm^-1, volumes, lumped masses),
 * surface primitives, marker weights and the tet patches, allocates all
 * device state and leaves every pad at rest with pose 0. Blocking. */
int tac_create_batch(const tac_pad_desc* pads, const tac_params* params, int n_pads,
                     const tac_indenter_desc* indenters, int n_envs, int pads_per_env,
                     const tac_options* opts, void* stream, tac_handle* out);

/* Free all device and host resources of the batch (synchronises its work).
 * A service call; the paper has no counterpart. */
int tac_destroy_batch(tac_handle h);

/* Reset every pad to rest (x = X, v = 0) with the current indenter pose set
 * to pose6_dev (device [n_pads*6]): the start of an episode, x^0 and v^0 of
 * the time stepping of Eq. (varopt). */
int tac_reset(tac_handle h, const float* pose6_dev, void* stream);

/* Set the indenter pose the next tac_step moves to, per pad (the plugin
 * input of Sec. 3.3: the object's pose relative to the sensor).
 * pose6_dev: device [n_pads*6] (rotation vector, translation) or NULL;
 * twist6_dev: device [n_pads*6] (angular velocity, linear velocity) or NULL.
 * With pose6_dev NULL the target is the current pose advanced by h * twist
 * (translation += h v, rotation composed with exp(h w)); with both given the
 * pose is used and the twist ignored; both NULL is TAC_ERR_INVALID_ARG. */
int tac_set_indenter(tac_handle h, const float* pose6_dev, const float* twist6_dev, void* stream);

/* Solve one frame for every pad: move each indenter from its current pose to
 * its target pose and minimise E (Supp. A). Writes the per-pad status
 * (TAC_PAD_*) and iteration count to caller-owned device arrays
 * pad_status_dev [n_pads] and iters_dev [n_pads] (either may be NULL), then
 * v = (x - x^t) / h and the current pose becomes the target pose.
 * Each pad is solved whole by one CTA of a persistent launch that takes pads
 * from a queue, longest first: the order is by the pad's solve time in its
 * previous frame, then by its tet count. Results do not depend on the order. */
int tac_step(tac_handle h, int* pad_status_dev, int* iters_dev, void* stream);

/* Adjoint of the last frame (gradients for calibration; the paper itself
 * calibrates with gradient-free CMA-ES, Sec. 4.2). At the frame's equilibrium
 * x* the gradient g vanishes on the free DOFs, so for a loss L of the
 * markers dL/dtheta = -lambda^T dg/dtheta with H lambda = dL/dx, H the exact
 * Hessian (mass + elastic + barrier + lagged friction). lambda is found by
 * block-Jacobi preconditioned CG with a matrix-free Hessian-vector product,
 * stopped at |r| <= tol |dL/dx| or max_iter iterations.
 * dL_dmarkers_dev: device [total_markers*2] float, dL/d(u_x, u_y) per marker
 *   in the layout of tac_markers.
 * dL_dtheta_dev: device [n_pads*9] double, per pad d L / d(Lame lambda,
 *   Lame mu, friction mu_f, rotation vector (3), translation (3)) of the
 *   indenter pose the frame ended at. kappa, eps_v, the frame's start state
 *   (x^t, v^t), its start pose and its friction lag are held fixed.
 * status_dev / iters_dev: device [n_pads] int (0 converged, 1 iteration cap,
 *   2 non-positive curvature d^T H d, 3 non-finite), PCG iterations; either
 *   may be NULL.
 * Must follow the tac_step whose frame is differentiated, with no other
 * state-changing call in between. */
int tac_adjoint(tac_handle h, const float* dL_dmarkers_dev, double* dL_dtheta_dev, int* status_dev,
                int* iters_dev, int max_iter, float tol, void* stream);

/* Adjoint of the last frame for a reverse sweep over a sequence of frames
 * (the multi-frame form of tac_adjoint; same method and stopping rule).
 * Each frame's friction lag (normal forces, contact normals, closest-point
 * weights, taken from the frame's start) is a constant of the frame, as it
 * is in the frame's solve; the frame's start then enters g only through
 * x-hat = x^t + h v^t (Eq. varopt) and the lagged friction displacement.
 * dL_dmarkers_dev: device [total_markers*2] float or NULL, as in tac_adjoint.
 * dL_dx_dev: device [total_verts*3] float or NULL, the loss gradient with
 *   respect to the frame's end positions beyond the markers (from later
 *   frames), in the caller vertex order of tac_get_state.
 * dL_dtheta_dev: device [n_pads*15] double, per pad d L / d(Lame lambda,
 *   Lame mu, mu_f, end pose rotation vector (3), end pose translation (3),
 *   start pose rotation vector (3), start pose translation (3)).
 * dL_dx0_dev, dL_dv0_dev: device [total_verts*3] float or NULL, caller
 *   order: dL/dx^t = (M + H_D) lambda and dL/dv^t = h M lambda, H_D the
 *   lagged friction Hessian; 0 on Dirichlet vertices.
 * status_dev / iters_dev / max_iter / tol: as in tac_adjoint.
 * lag_mode: 0 holds the lag fixed as above; 1 differentiates it as a
 *   function of the frame's start state and start pose, which makes a
 *   reverse sweep the total derivative of a run whose frames each lag
 *   themselves. dL/dx^t and the start-pose entries then gain
 *   -d(lambda^T g)/d(start) through the lag, from float64 central
 *   differences of each lagged pair's friction force rebuilt from its
 *   primitives' start positions (1e-10 m, 1e-7 rad).
 * A sweep over frames 1..F gives frame f's end state the gradient
 *   (markers of frame f) + a_x + a_v / h with a_x, a_v from frame f+1, then
 *   passes a_x = dL/dx^t - a_v / h and a_v = dL/dv^t to frame f-1 (since
 *   v^f = (x^f - x^(f-1)) / h). Must follow the tac_step of the frame. */
int tac_adjoint_frame(tac_handle h, const float* dL_dmarkers_dev, const float* dL_dx_dev, double* dL_dtheta_dev,
                      float* dL_dx0_dev, float* dL_dv0_dev, int* status_dev, int* iters_dev, int max_iter, float tol,
                      int lag_mode, void* stream);

/* Install a frame that was solved before (by a tac_step from the start
 * state x0, v0 at pose_start to pose_end, ending at x1) so that tac_adjoint
 * or tac_adjoint_frame can differentiate it without solving it again, as a
 * reverse sweep over saved frames needs. The frame's friction lag is
 * rebuilt from the start state and pose by the steps of tac_step's frame
 * setup, so it equals the lag of the original solve when that solve started
 * from this state (a tac_set_state of x0, v0 after a tac_reset at
 * pose_start). The batch is left at the end state: positions x1, velocities
 * (x1 - x0) / h, current pose pose_end.
 * x0_dev, v0_dev, x1_dev: device [total_verts*3] float, caller vertex order;
 * pose_start_dev, pose_end_dev: device [n_pads*6] float. */
int tac_set_frame(tac_handle h, const float* x0_dev, const float* v0_dev, const float* pose_start_dev,
                  const float* x1_dev, const float* pose_end_dev, void* stream);

/* Marker displacement field (u_x, u_y) per marker of every pad, in pad order:
 * out_dev: device [sum_p n_markers(p) * 2] float (Sec. 3.2). */
int tac_markers(tac_handle h, float* out_dev, void* stream);

/* Copy the vertex state out / in: x_dev, v_dev device [total_verts*3] float
 * (positions and velocities, pads concatenated in order): the x^t and v^t
 * that the next frame's x-hat = x^t + h v^t of Eq. (varopt) is built from,
 * and the per-frame checkpoints of a multi-frame adjoint. tac_set_state
 * keeps the current pose. */
int tac_get_state(tac_handle h, float* x_dev, float* v_dev, void* stream);
int tac_set_state(tac_handle h, const float* x_dev, const float* v_dev, void* stream);

/* Replace the material / solver parameters of all pads (host [n_pads]):
 * the per-environment material randomisation of Supp. C and the candidate
 * (E, nu, rho, mu_f) of a calibration step (Sec. 4.2). */
int tac_set_params(tac_handle h, const tac_params* per_pad, int n);

/* The parameters in effect per pad (host [n]): as last set, with kappa and
 * eps_v resolved to the values the solve uses (their defaults filled in). */
int tac_get_params(tac_handle h, tac_params* per_pad, int n);

/* Candidate contact set (the set C of Eq. ipc_energy) of one pad for given
 * positions: every (type, i, j) whose gel-primitive AABB inflated by r
 * overlaps the indenter-primitive AABB, decided in float64 on the float32
 * inputs. type 0 = gel vertex i x indenter triangle j; 1 = gel surface
 * triangle i x indenter vertex j; 2 = gel surface edge i x indenter edge j
 * (canonical surface order: boundary faces with sorted vertex ids, sorted;
 * distinct surface edges (lo, hi), sorted; indenter edges likewise).
 * x_dev: device [n_verts(pad)*3] gel positions; y_dev: device
 * [n_indenter_verts*3] indenter world vertices; pairs_out_dev: device
 * [capacity*3] int, sorted lexicographically; count_dev: device int, the
 * full count (entries beyond capacity are not written). */
int tac_broadphase(tac_handle h, int pad, const float* x_dev, const float* y_dev, double r,
                   int* pairs_out_dev, int capacity, int* count_dev, void* stream);

/* Allocation-free candidate search (the paper has no counterpart; this is
 * a service for callers of the library). It returns the same candidate set
 * as tac_broadphase, for callers that cannot allocate device memory: code
 * running while a stream is being captured into a CUDA graph, real-time or
 * embedded loops whose memory is fixed before they start, and hosts that
 * give the library no allocator. It takes no batch handle; the caller
 * passes every input and output as device arrays, and the call allocates and
 * frees nothing (no cudaMalloc, cudaFree or library allocator).
 * Inputs: x_dev gel positions [n*3]; the gel surface primitives in the
 * canonical order described at tac_broadphase (vertex ids [n_surf_verts],
 * triangles [n_surf_tris*3], edges [n_surf_edges*2]); y_dev indenter world
 * vertices [n_ind_verts*3], indenter triangles [n_ind_tris*3] and distinct
 * sorted edges [n_ind_edges*2]; the inflation radius r. Outputs:
 * pairs_out_dev [capacity*3] (type, i, j) triples sorted lexicographically,
 * count_dev the full count (entries beyond capacity are not written).
 * Scratch: one fixed array of 65536 16-byte slots (1 MiB) built into the
 * library; every GPU that loads the library holds it until the process
 * exits. A call needs ceil((n_ind_tris + n_ind_verts + n_ind_edges) / 4) +
 * capacity slots; a larger request fails with TAC_ERR_INVALID_ARG before any
 * device work. Each scratch entry a call reads is written earlier by the
 * same call, so the contents left by the previous call need no clearing.
 * Preconditions the call does not check: every id in surf_verts_dev,
 * surf_tris_dev and surf_edges_dev is below the number of vertices in x_dev,
 * and every id in ind_tris_dev and ind_edges_dev is below n_ind_verts; an id
 * out of range reads outside the caller's arrays.
 * The first call on a device looks up the device address of the array and
 * sets the kernel's shared-memory limit: make that first call before any
 * stream capture. The address is kept per device ordinal for the life of the
 * process; after a cudaDeviceReset it is stale and the library must not be
 * called on that device again. All calls share the one array, so calls whose GPU work
 * overlaps (different streams or threads on one device) race on it and must
 * be serialised by the caller. */
int tac_broadphase_static(const float* x_dev, const int* surf_verts_dev, int n_surf_verts,
                          const int* surf_tris_dev, int n_surf_tris, const int* surf_edges_dev,
                          int n_surf_edges, const float* y_dev, int n_ind_verts, const int* ind_tris_dev,
                          int n_ind_tris, const int* ind_edges_dev, int n_ind_edges, double r,
                          int* pairs_out_dev, int capacity, int* count_dev, void* stream);

/* Verification entry point: evaluate the pieces of one PNCG iteration for
 * every pad at displacement u (x = X + u) along direction p with the
 * indenter at its current pose, inertia centred at u (xhat = x) and no
 * friction lag. Inputs u_dev, p_dev: device [total_verts*3] float.
 * Outputs (device, any may be NULL):
 *   grad_dev  [total_verts*3]  float  gradient at u + alpha p
 *   blk_dev   [total_verts*6]  float  diagonal blocks at u + alpha p
 *                                     (xx, yy, zz, xy, xz, yz)
 *   scal_dev  [n_pads*8]       double (p^T H p: elastic, contact, inertia;
 *             E(u + alpha p) - E(u): total; alpha_ccd; min distance at u;
 *             number of candidate pairs; max |g_i| at u + alpha p) */
int tac_debug_eval(tac_handle h, const float* u_dev, const float* p_dev, float alpha,
                   float* grad_dev, float* blk_dev, double* scal_dev, void* stream);

/* Per-pad counters of the last tac_step (device [n_pads*16] long long):
 * iterations, substeps, broad-phase rebuilds, Armijo halvings, tet passes,
 * vertex passes, pair evaluations, peak candidate count, then nanoseconds
 * spent in: p^T H p tet passes, gradient tet passes, contact p^T H p and
 * step bound, contact gradient passes, vertex passes, indenter advance and
 * rebuilds, frame setup, and the whole pad solve. */
int tac_stats(tac_handle h, long long* stats_dev, void* stream);

/* Convergence record of the last tac_step per pad (device [n_pads*4]
 * double): final max |g_i|, the stopping target, g_ref of the frame, and the
 * largest force component F summed into the float32 gradient (elastic
 * per-corner forces, barrier and friction per-slot forces). The target is
 * max(tol * g_ref, floor_ulps * 2^-24 * F) (tac_params.floor_ulps, 256 by
 * default): a float32 gradient is not resolved below a few hundred ulps of
 * the forces summed into it. */
int tac_pad_norms(tac_handle h, double* norms_dev, void* stream);

/* Host only (no device work, no handle): the marker map that tac_create_batch
 * builds for this pad under marker_mode (see tac_params). ids_host and w_host
 * are caller-owned host arrays of [n_markers*4]: marker m reads vertices
 * ids_host[4m..4m+3] (input vertex ids) with weights w_host[4m..4m+3]; the
 * barycentric map fills three slots and gives the fourth weight 0 (its id
 * repeats the first). Validates the mesh like tac_create_batch
 * (TAC_ERR_INVALID_MESH with a message). tac_markers and the adjoint's
 * right-hand side read the pads through this map. */
int tac_marker_map(const tac_pad_desc* pad, int marker_mode, int* ids_host, float* w_host);

/* Host only (no device work, no handle): how tac_create_batch lays out this
 * pad's mesh: the number of 32-tet warp patches, of colour classes (patches
 * of one class share no vertex), of rest-shape classes in its Dm^-1 table
 * (0 when the mesh needs more than 32 and streams one Dm^-1 per tet; see
 * tac_options.no_dm_table), and the largest deviation of a tet's Dm^-1 from
 * its class representative, relative to the representative's largest entry
 * (at most 1e-5 by construction), the rounds a scatter pass takes (a colour
 * class costs ceil(patches / 8), one patch per warp) and the number of
 * vertices that two patches of one class share (0 for a valid layout: the
 * scatter passes rely on it). Any output pointer may be NULL. Validates the
 * mesh like tac_create_batch (TAC_ERR_INVALID_MESH with a message). */
int tac_mesh_info(const tac_pad_desc* pad, int* n_patches, int* n_colours, int* n_dm_types, double* dm_dev,
                  int* n_rounds, int* n_conflicts);

/* Sizes: total vertices, total markers, candidate capacity per pad, and the
 * number of CTAs of one tac_step launch (resident CTAs of the device, at most
 * one per pad). A service call for sizing caller buffers; the paper has no
 * counterpart. Any output pointer may be NULL. */
int tac_sizes(tac_handle h, int* total_verts, int* total_markers, int* pair_capacity, int* grid_ctas);

/* Block shape of tac_step's persistent solve launch. threads = 256: one
 * 256-thread CTA per pad, two CTAs per SM (the default); 512: one 512-thread
 * CTA per pad, one per SM, so that each phase of a pad's solve (the
 * colour-class rounds of the tet passes, the pair and vertex passes) spreads
 * over twice the threads: the shape for batches with fewer pads than the
 * 256-thread shape has CTA slots (Sec. 5.1 measures throughput against the
 * number of environments). Each shape is deterministic and independent of the
 * pads' order; the two differ in the order of their block reductions, so
 * their results agree to rounding, not bit for bit. TAC_ERR_INVALID_ARG for
 * any other value. No device work. */
int tac_set_block_shape(tac_handle h, int threads);

/* Autotuner of the block shape. From the current state it solves the next
 * frame (indenter poses pose6_dev, device [n_pads*6]) reps times in each
 * shape, each time from the same saved state, times each solve with CUDA
 * events on `stream`, puts back the state, the poses and the per-pad records
 * the schedule keys on, and selects the shape of the smaller mean time (as
 * tac_set_block_shape). threads_out (host) receives the chosen shape; ms_out
 * (host [2], may be NULL) the mean milliseconds of the 256- and 512-thread
 * solves. The tuning solves count as the last tac_step for tac_stats,
 * tac_pad_norms and tac_adjoint: call it before a tac_step, not between a
 * tac_step and its adjoint. Allocates scratch for one copy of the state
 * (freed before it returns) and synchronises the stream. */
int tac_autotune_block_shape(tac_handle h, const float* pose6_dev, int reps, int* threads_out, float* ms_out,
                             void* stream);

/* Message of the last error on this thread (static storage, never NULL). */
const char* tac_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TAC_H_ */
