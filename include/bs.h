/*
 * bs.h -- C ABI of libbs: Biot-Savart velocity on tetrahedral meshes with
 * linearly varying nodal vorticity, on one GB300 GPU (sm_103a).
 *
 * Method (Carley, "Evaluation of Biot-Savart integrals on tetrahedral
 * meshes"): for every evaluation point x and every tetrahedron T,
 *   v(x) += contribution of T to  -(1/4pi) int r x omega / R^3 dV   (Eq. 1)
 *   - T far  (|x - centroid(T)|^2 > (far_ratio * circumradius(T))^2):
 *       tet Gauss rule applied to Eq. 1 (Section 1);
 *   - T near: ray rule of Section 2 -- for each direction s_nm of the
 *       Gauss-Legendre product rule of Eq. 3, the chord [R0, R1] of the line
 *       x + R s through T and the exact integral of the linear omega along
 *       it (Eq. 5, with the factor sign(R) that Eq. 2 needs when theta
 *       covers [0, pi] only), weighted by k_nm = (pi/16) sin(phi_n) w_n w_m.
 *       With near_rule = BS_NEAR_EXACT the near tets take instead the exact
 *       integral of Eq. 1 over the tet (the analytic near-field evaluation
 *       Section 1 compares the ray rule against).
 *
 * Conventions for every call:
 *   - Arrays are row-major and tightly packed: points/nodes/omega/velocity
 *     are [count][3] float64, tets are [count][4] int32 node indices.
 *   - "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *     global memory of the current device.  The caller owns every array it
 *     passes; the library copies what it keeps.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream are asynchronous and stream-ordered;
 *     they do not synchronise the host.
 *   - Every call returns BS_OK (0) or one of the BS_ERR_* codes below and,
 *     on error, leaves a message for bs_last_error() (per host thread).
 *     A call that returns an error has launched no kernel and written no
 *     output.
 */
#ifndef BS_H
#define BS_H

#include <stdint.h>

#if defined(__GNUC__)
#define BS_API __attribute__((visibility("default")))
#else
#define BS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define BS_OK 0
#define BS_ERR_ARG 1     /* NULL pointer, negative size, parameter out of range */
#define BS_ERR_MESH 2    /* node index out of range, or |volume| <= 1e-14 h^3   */
#define BS_ERR_ORDER 3   /* tet_gauss_order not in {1, 4, 8, 27, 64}            */
#define BS_ERR_CUDA 4    /* a CUDA runtime call failed                          */
#define BS_ERR_TIMEOUT 5 /* a bounded device-side wait gave up                  */

#define BS_FP64 0 /* every step in float64                                           */
#define BS_FP32 1 /* float32 bulk with compensated per-point sums; the ray steps of   */
                  /* pairs whose point sits on a vertex, edge or face of the tet run  */
                  /* in float64; the final per-point sum is float64                   */

#define BS_NEAR_RAY 0   /* near tets by the ray rule of Section 2 (the paper's method)      */
#define BS_NEAR_EXACT 1 /* near tets by the exact integral of Eq. 1 over the tet (the       */
                        /* analytic near-field evaluation Section 1 compares against:       */
                        /* face and edge integrals in closed form, 6 logarithms and 12      */
                        /* atan2 per tet) with float64 geometry; the logarithms and arc     */
                        /* tangents in float64 (BS_FP64) or float32 (BS_FP32); no ray hits   */
                        /* are counted                                                      */

typedef struct bs_ctx *bs_handle;
typedef struct bs_batch_ctx *bs_batch;

typedef struct {
    double far_ratio;    /* far <=> |x-c|^2 > (far_ratio*rho)^2; must be >= 2 (so a tet
                            with x at a vertex is never far) or +INFINITY (every tet
                            near: the paper's all-ray rule of Section 2.2)          */
    int tet_gauss_order; /* far rule points: 1 (centroid), 4 (degree 2), 8/27/64
                            (conical product rules of degree 3/5/7)                 */
    int n_theta;         /* M Gauss points in theta (azimuth over [0, pi]), 1..256   */
    int n_phi;           /* N Gauss points in phi (polar, weighted by sin phi), 1..256 */
    int precision;       /* BS_FP64 or BS_FP32                                       */
    int32_t *counts;     /* optional device [k][3] int32 output: near tets, far tets,
                            ray hits (line-tet pairs with chord > 1e-9 * longest edge);
                            NULL to skip                                             */
    int near_rule;       /* BS_NEAR_RAY (0) or BS_NEAR_EXACT (1)                      */
} bs_params;

/* Upload a mesh and precompute its per-tet tables (Section 2.2 steps 2-3 and
 * the far-rule data).  nodes: host [n_nodes][3]; tets: host [n_tets][4];
 * omega: host [n_nodes][3].  Tets of either orientation are accepted.
 * Synchronises the device.  Errors: BS_ERR_ARG (NULL, n_nodes < 1,
 * n_tets < 0), BS_ERR_MESH (index out of range or degenerate tet; the
 * message names the first offending tet), BS_ERR_CUDA.  On success *out
 * owns every device buffer of the mesh until bs_destroy. */
BS_API int bs_create(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets, const double *omega,
              bs_handle *out);

/* Replace node positions and/or nodal vorticity (same connectivity) from
 * device arrays [n_nodes][3] (either may be NULL to keep the current one)
 * and recompute the per-tet tables on `stream` (one step of a Lagrangian vortex method, Section 1).
 * Asynchronous: a degenerate tet is reported by the next bs_status. */
BS_API int bs_update(bs_handle h, const double *nodes_dev, const double *omega_dev, void *stream);

/* Velocity at k evaluation points.  eval_pts_dev: device [k][3];
 * out_dev: device [k][3], overwritten (not accumulated).  k = 0 is a no-op.
 * Errors: BS_ERR_ARG, BS_ERR_ORDER, BS_ERR_CUDA. */
BS_API int bs_velocity(bs_handle h, const double *eval_pts_dev, int64_t k, const bs_params *p, double *out_dev,
                void *stream);

/* Same as bs_velocity with HOST buffers: copies the points in, evaluates and
 * copies the velocities out on `stream`, then synchronises it. */
BS_API int bs_velocity_host(bs_handle h, const double *eval_pts_host, int64_t k, const bs_params *p, double *out_host,
                     void *stream);

/* Velocity at the handle's own nodes (the evaluation points of the Lagrangian
 * method, Section 1): out_dev [n_nodes][3] (device, overwritten), p->counts
 * optional ([n_nodes][3]).  Same result as bs_velocity at the nodes.  With
 * far_ratio = +inf (every pair by the ray rule, Eq. 2-5) and at most 4096
 * directions, every line through a node is traced through the mesh by face
 * neighbours (the tracing through the mesh that the paper's conclusion, §4,
 * proposes): from the node, each half-line crosses the tets it meets one after
 * the other until it leaves the mesh, each tet adding its chord of Eq. 5.
 * The walk is used with the ray near rule (p->near_rule = BS_NEAR_RAY) when
 * the mesh is conforming (a face belongs to at most two tets, every node to
 * some tet) and not folded (no two tets sharing a face on the same side of
 * it, checked on the device after each change of the node positions);
 * otherwise the call evaluates the nodes as bs_velocity does.  On a convex domain every line leaves the mesh once; on a
 * non-convex one (checked on the device after each change of the node
 * positions: some boundary node outside some boundary face's plane) a line
 * that leaves is followed through a uniform grid of the boundary faces to
 * where it comes back in, if it does.  The first such call builds the face
 * adjacency and the node-to-tet incidence on the host (synchronous, once per
 * handle; about 200 bytes per tet and 100 per boundary face of device memory,
 * owned by the handle); later calls are asynchronous on `stream`.  A walk that exceeds max(4096, 64 n_tets^(1/3))
 * tets (impossible on a valid mesh) stops and raises BS_ERR_TIMEOUT at the next
 * bs_status.  With a finite far_ratio (the hybrid rule) and the ray near
 * rule, when the kernel variant in use leaves the near pairs to a pass of
 * their own (see bs_variant_shape), the far rule runs as in bs_velocity and
 * the near field is taken by the same walk, restricted to the tets the far
 * rule's test calls near (the same decision, bit for bit): a half-line
 * stops once it is farther from the node than max over tets of (far_ratio
 * circumradius + the tet's bounding radius about its centroid), beyond
 * which every tet is far.  On a mesh the walk cannot serve, the near pass
 * evaluates the near pairs instead.  Setting the environment variable
 * BS_WALK=0 disables the walk.  Errors: BS_ERR_ARG, BS_ERR_ORDER,
 * BS_ERR_CUDA. */
BS_API int bs_velocity_nodes(bs_handle h, const bs_params *p, double *out_dev, void *stream);

/* Velocity at the nodes (as bs_velocity_nodes) and its derivative along a
 * direction per node: dout_dev[i] = (e_i . grad) v at node i, with e_i =
 * dirs_dev[i] ([n_nodes][3] device, or NULL for the nodal vorticity, which
 * makes dout the stretching term (omega . grad) v of the vorticity equation;
 * the paper gives no vorticity update).  Defined for the all-ray method
 * (far_ratio = +inf, at most 4096 directions): along each line the rule
 * integrates the piecewise-linear vorticity omega_h (zero outside the mesh),
 * and the derivative is the chord length in each tet the line crosses times
 * e . grad omega in that tet, plus the jump of omega to zero where the line
 * leaves the mesh (omega there times the shift of the exit point), computed
 * during the mesh walk.  At a node on the mesh boundary the rule is not
 * differentiable (omega jumps at the node itself); the value returned there
 * leaves out the jump at the node.  Other parameters (including
 * near_rule = BS_NEAR_EXACT) return BS_ERR_ARG; a mesh the walk cannot serve
 * (not conforming, or folded) gets the velocity but no derivative, reported as
 * BS_ERR_MESH by the next bs_status.
 * Asynchronous on `stream` after the first call (see bs_velocity_nodes). */
BS_API int bs_velocity_nodes_dderiv(bs_handle h, const bs_params *p, const double *dirs_dev, double *out_dev,
                                    double *dout_dev, void *stream);

/* One Heun step of the node positions and the nodal vorticity with vortex
 * stretching: dx/dt = v, d omega/dt = (omega . grad) v at the nodes, both from
 * bs_velocity_nodes_dderiv (all-ray method only, see there):
 *   (v0, s0) at (x0, omega0); x* = x0 + dt v0, omega* = omega0 + dt s0;
 *   (v1, s1) at (x*, omega*); x1 = x0 + dt (v0 + v1)/2,
 *   omega1 = omega0 + dt (s0 + s1)/2.
 * The handle's nodes and vorticity become (x1, omega1).  p->counts must be
 * NULL.  The first call allocates six [n_nodes][3] work arrays owned by the
 * handle.  Asynchronous on `stream`. */
BS_API int bs_rk2_step_stretch(bs_handle h, double dt, const bs_params *p, void *stream);

/* One Heun (RK2) step of the Lagrangian vortex method (Section 1: the nodes
 * move with the flow and the velocity is re-evaluated on the moved mesh):
 *   v0 = v(x0) at the nodes;  x* = x0 + dt v0;  v1 = v(x*) at the moved nodes;
 *   x1 = x0 + dt (v0 + v1) / 2.
 * Every velocity evaluation is bs_velocity_nodes with parameters p
 * (p->counts must be NULL); the connectivity and the nodal vorticity stay
 * fixed (no vortex stretching: the paper gives no vorticity update).  The
 * handle's node positions become x1.  Asynchronous on `stream`; a tet that
 * the motion made degenerate is reported by the next bs_status.  The first
 * call allocates three [n_nodes][3] work arrays owned by the handle. */
BS_API int bs_rk2_step(bs_handle h, double dt, const bs_params *p, void *stream);

/* n_steps Heun steps: bs_rk2_step (stretch = 0) or bs_rk2_step_stretch
 * (stretch = 1) repeated, with the same results bit for bit.  The first step
 * runs as a plain call; the second is captured as a CUDA graph on a stream of
 * the handle (joined to `stream` by events) and the graph is launched for the
 * remaining steps, which removes the host cost of the step's ~25 launches.
 * The steps run one by one instead when n_steps <= 1, while bs_profile is on,
 * or when the capture does not succeed.  Asynchronous on `stream`; the first
 * call creates the handle's stream and two events.  Errors: as bs_rk2_step,
 * and BS_ERR_ARG for n_steps < 0 or stretch not 0/1. */
BS_API int bs_rk2_steps(bs_handle h, double dt, int64_t n_steps, int stretch, const bs_params *p, void *stream);

/* Number of steps bs_rk2_steps has run by graph launch on this handle. */
BS_API int bs_graph_steps(bs_handle h, int64_t *steps);

/* Copy the handle's current node positions to device array nodes_dev [n_nodes][3]. */
BS_API int bs_nodes(bs_handle h, double *nodes_dev, void *stream);

/* Copy the handle's current nodal vorticity to device array omega_dev [n_nodes][3]
 * (it changes under bs_update and bs_rk2_step_stretch). */
BS_API int bs_omega(bs_handle h, double *omega_dev, void *stream);

/* Synchronise `stream` and return BS_ERR_MESH / BS_ERR_TIMEOUT if a kernel of
 * this handle raised its device error flag since the last call (clears it). */
BS_API int bs_status(bs_handle h, void *stream);

/* Limits of the handle's bounded device waits, and a test of their give-up
 * path (the paper has no counterpart).  Every device wait of the library is
 * bounded: a mesh walk stops after a number of tets per half-line, and the
 * velocity and all-ray kernels stop waiting for a bulk copy of a tet tile
 * after a number of polls; either then raises the handle's error flag, the
 * kernel returns, and the next bs_status reports BS_ERR_TIMEOUT.
 *   walk_max_steps  > 0: tets a half-line may cross (0: the default,
 *                   max(4096, 64 n_tets^(1/3)) capped at n_tets);
 *   copy_wait_polls > 0: polls of a bulk-copy wait (0: the default, 2^26,
 *                   about a second);
 *   withhold_copies = 1: the velocity and all-ray kernels arm their copy
 *                   barriers but issue no copy, so every wait runs out (a
 *                   test of the give-up path: no copy is ever in flight, so
 *                   nothing can land after the kernel returned).  Results are
 *                   then meaningless; 0 restores normal operation.
 * On a valid mesh with the defaults no limit is ever reached.  A kernel that
 * gives up first waits (with the same bound) for its own copies still in
 * flight.  The settings apply to the calls on this handle that follow.
 * Errors: BS_ERR_ARG (NULL handle, negative limit, withhold_copies not 0/1). */
BS_API int bs_set_wait_limits(bs_handle h, int64_t walk_max_steps, int64_t copy_wait_polls, int withhold_copies);

/* Free every device buffer of the handle (synchronises the device). */
BS_API int bs_destroy(bs_handle h);

/* Mesh sizes of a handle. */
BS_API int bs_mesh_size(bs_handle h, int64_t *n_nodes, int64_t *n_tets);

/* Velocity at k points without allocating any device memory.  The paper has
 * no counterpart: this is a deployment variant for callers that must not let
 * a library allocate GPU memory (an application whose memory is all handed
 * out by its own pool under a fixed budget, or a time-critical loop that
 * cannot take the device synchronisation or the out-of-memory failure of a
 * driver allocation).  Nothing is created beforehand: the mesh comes straight
 * from device arrays nodes_dev [n_nodes][3], tets_dev [n_tets][4] (int32),
 * omega_dev [n_nodes][3]; eval_pts_dev [k][3] and out_dev [k][3] as in
 * bs_velocity (out overwritten), p->counts optional.  Every table and partial
 * sum lives in one fixed array of device memory owned by the library (about
 * 11 MB, present on every GPU that loads the library until the process
 * exits), so the sizes are capped: n_tets <= 8192, k <= 4096,
 * n_theta * n_phi <= 4096, tet_gauss_order 1 or 4; larger requests return
 * BS_ERR_ARG (BS_ERR_ORDER for the rule) before any work is queued.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current): make that first call before any stream
 * capture.  All calls share the one array, which keeps the last call's
 * contents: two calls whose work overlaps on the GPU (different streams, or
 * different host threads, without ordering between them) race and give
 * wrong results; order them on one stream.  The mesh is not validated on
 * the host (that would need a synchronisation): a node index out of range,
 * a degenerate tet (|volume| <= 1e-14 h^3) or a bulk-copy wait that gave up
 * is found on the device, and the call's last kernel then overwrites every
 * velocity with NaN and every count with -1 (use bs_create to validate a
 * mesh beforehand). */
BS_API int bs_velocity_noalloc(const double *nodes_dev, int64_t n_nodes, const int32_t *tets_dev, int64_t n_tets,
                               const double *omega_dev, const double *eval_pts_dev, int64_t k, const bs_params *p,
                               double *out_dev, void *stream);

/* The error state of the last bs_velocity_noalloc call on the current
 * device, read from the library's fixed array (no allocation).  The read is
 * queued on `stream` (a cudaStream_t, NULL = the legacy default stream) and
 * the call synchronises that stream, so it sees every bs_velocity_noalloc
 * call queued before it there.  Returns BS_OK if that call found nothing
 * wrong (or no call has run on this device yet); BS_ERR_MESH for a node index
 * out of range or a degenerate tet, with *first_bad_tet (optional, may be
 * NULL; -1 when there is no error) the lowest such tet; BS_ERR_TIMEOUT for a
 * bulk-copy wait that gave up; BS_ERR_CUDA if the read failed.  The state is
 * shared by every call on the device: with calls on several unordered
 * streams it belongs to whichever call wrote it last.  Calling this does
 * not clear it; the next bs_velocity_noalloc call does. */
BS_API int bs_noalloc_status(void *stream, int64_t *first_bad_tet);

/* Kernel timing of a handle (for benchmarks).  bs_profile(h, 1) starts
 * recording a CUDA event pair around every velocity-kernel launch of this
 * handle (on the launch stream) and counting every kernel the handle
 * launches; bs_profile(h, 0) stops.  bs_profile_read synchronises the device
 * and returns the summed velocity-kernel time (ms), the number of velocity
 * kernel launches and the number of all kernel launches since profiling was
 * enabled. */
BS_API int bs_profile(bs_handle h, int enable);
BS_API int bs_profile_read(bs_handle h, double *kernel_ms, int64_t *kernel_launches, int64_t *all_launches);

/* Message of the last error on the calling host thread ("" if none). */
BS_API const char *bs_last_error(void);

/* Tables computed on the device, copied to host arrays (synchronous):
 * directions s [n_phi*n_theta][3] and weights k [n_phi*n_theta] of Eq. 3,
 * line index l = n*n_theta + m;  tet rule barycentric points [order][4] and
 * weights [order] (fractions of |V|). */
BS_API int bs_direction_table(int n_phi, int n_theta, double *s_host, double *k_host);

BS_API int bs_tet_rule(int order, double *bary_host, double *w_host);

/* Many meshes in one persistent launch (evaluation points = each mesh's own
 * nodes).  bs_batch_create: host array of n handles (not owned; they must
 * outlive the batch).  bs_batch_velocity: outs[i] is a device [n_nodes_i][3]
 * output for mesh i (host array of n device pointers); p->counts must be NULL.
 * The work queue is built on the device; the launch sequence is captured once
 * into a CUDA graph per (params, stream) and replayed (on the legacy default
 * stream it is launched directly).  With a variant that leaves the near pairs
 * out of the far kernel (the default for the ray rule), each mesh's near field
 * is taken by its mesh walk, as in bs_velocity_nodes, where the mesh allows it
 * (the first call builds each mesh's walk tables on the host and synchronises),
 * else by one near pass over the points of every such mesh.  The meshes' walks
 * run concurrently on 8 non-blocking side streams the batch owns (created by
 * the first call that walks, destroyed by bs_batch_destroy), alongside the far
 * kernel, which they do not depend on: they wait on an event recorded on
 * `stream` before it, and `stream` waits on each of them before the near pass,
 * so the call is ordered on `stream` alone. */
BS_API int bs_batch_create(const bs_handle *meshes, int n, bs_batch *out);
BS_API int bs_batch_velocity(bs_batch b, const bs_params *p, double *const *outs, void *stream);
/* Synchronise `stream` and report a device error of the batch's launches since
 * the last call: BS_ERR_TIMEOUT if a bounded wait of the batched far kernel
 * gave up (the batch follows the wait limits bs_set_wait_limits gave its first
 * mesh), else the first error bs_status reports for its meshes (their tables
 * and near walks); every flag read is cleared. */
BS_API int bs_batch_status(bs_batch b, void *stream);
BS_API int bs_batch_destroy(bs_batch b);

/* Kernel variants and the autotuner (the paper has no counterpart: launch
 * shapes of this GPU implementation).
 *
 * The velocity kernel is compiled in several variants per (precision, tet
 * rule, near rule), each a launch shape: evaluation points per thread, tets
 * per shared-memory tile, pipeline stages, CTAs per SM its registers are
 * budgeted for, how the near pairs are drained (routine called, inlined, or
 * inlined with the pair's state in shared memory), ray bundle (lines each
 * lane takes per iteration of the ray rule), how the far sweep pairs values
 * in its packed float32x2 registers (two quadrature points, or two
 * evaluation points), and the unroll of the far sweep's tet loop.  Every
 * variant computes the same rule; results differ only by rounding.
 *
 * Which variant a bs_velocity call uses: the environment variable BS_VARIANT
 * if set (every call), else the variant pinned by bs_set_variant, else the
 * autotuner's cache entry for this GPU (name and SM count), precision, tet
 * rule, near rule, direction count and size class (ceil(log2) of the point
 * and tet counts, and whether the points are the nodes of bs_velocity_nodes),
 * else, for the ray rule: at the nodes (at most 4096 directions) the first
 * variant that leaves the near pairs to the mesh walk -- the one with one
 * point per thread on a mesh too small to fill the GPU with variant 0's work
 * items (fewer than 8 GPU-fulls); elsewhere, on such a small mesh, the
 * variant with one point per thread that drains the near pairs in the far
 * kernel; else variant 0.  A batch uses BS_VARIANT, else its first mesh's
 * pinned variant, else (ray rule) variant 0 if it leaves the near pairs to
 * the near pass, else the one-point variant when every mesh has at most
 * 80000 tets, else variant 0.
 *
 * The cache is a JSON file: entries are read from tune_cache.json beside the
 * package directory (shipped, written by bs_autotune on this GPU model) and
 * from the file named by the environment variable BS_TUNE_CACHE, whose
 * entries take precedence. */

/* Number of variants for a precision, tet rule and near rule. */
BS_API int bs_num_variants(int precision, int tet_gauss_order, int near_rule, int *n);
/* Launch shape of a variant: shape[0..7] = points per thread, tets per tile,
 * pipeline stages, CTAs per SM of the register budget, near-pair drain
 * (0 routine called, 1 inlined, 2 inlined with the pair's state in shared
 * memory), ray bundle (lines per lane per iteration), far sweep pairing two
 * evaluation points (1) or two quadrature points (0), unroll of the far
 * sweep's tet loop. */
BS_API int bs_variant_shape(int precision, int tet_gauss_order, int near_rule, int variant, int32_t *shape);
/* Pin a variant for this handle's calls with this precision, tet rule and
 * near rule (-1 restores the automatic choice).  Errors: BS_ERR_ARG (variant
 * out of range), BS_ERR_ORDER. */
BS_API int bs_set_variant(bs_handle h, int precision, int tet_gauss_order, int near_rule, int variant);

/* Choose the variant for this mesh's own nodes and the parameters p: if the
 * cache holds an entry for this GPU and problem (see above), take it without
 * timing; else time every variant on `stream` (each after a warm-up call),
 * take the fastest, and store it in the cache (in BS_TUNE_CACHE if set, else
 * the shipped file, when the file is writable; for this process in any case).
 * The environment variable BS_TUNE_FORCE=1 times even on a cache hit.  Two
 * paths are tuned, each with its own cache entry: bs_velocity at the nodes
 * (the points path) and, for the hybrid rule with the ray near rule,
 * bs_velocity_nodes (the nodes path, where the mesh walk can take the near
 * field).  Calls that run the all-ray kernel (far_ratio = +inf, at most 4096
 * directions, the ray rule) have a single launch shape and need no tuning.
 * Synchronises the stream; allocates and frees one [n_nodes][3] output. */
BS_API int bs_autotune(bs_handle h, const bs_params *p, void *stream);
/* The variant the last bs_autotune for this precision and tet rule (ray
 * near rule) chose or found in the cache for the points path (at_nodes = 0:
 * bs_velocity) or the nodes path (at_nodes = 1: bs_velocity_nodes); 0 if
 * none. */
BS_API int bs_tuned_variant(bs_handle h, int precision, int tet_gauss_order, int at_nodes, int *variant);

#ifdef __cplusplus
}
#endif
#endif /* BS_H */
