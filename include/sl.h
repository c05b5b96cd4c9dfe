/*
 * sl.h -- C ABI of the GB300 library for the explicit semi-Lagrangian spectral (DSEM-SL)
 * transport step of Natarajan & Jacobs, "An explicit semi-Lagrangian, spectral method for
 * solution of Lagrangian transport equations in Eulerian-Lagrangian formulations"
 * (arXiv:1910.06476).
 *
 * One call of sl_step advances every element of a mesh by one time step (Sec. 4):
 *   (a) particles are seeded at the element's Gauss nodes (Sec. 4.1, eq. gaussquad, 4.2);
 *   (b) they are integrated explicitly through the velocity field together with the value
 *       equation D phi / Dt = -phi div u (Sec. 4.2, eq. 4.4a, 4.8; eq. 2.4, 2.5);
 *   (c) the advected polynomial is remapped to the Gauss nodes (eq. 4.9 in 1D, the
 *       collocation system eq. 5.4 in 2D) and its face traces are taken (eq. remap_bnd,
 *       2dx_bnd_interpolate, 2dy_bnd_interpolate);
 *   (d) a least-squares fit constrained by upwinded interface values (eq. 4.12a) and
 *       optionally by local mass and energy (eq. 4.14, quad, remap_mass, remap_energy)
 *       yields phi^{n+1} (eq. matrix_a).
 *
 * Conventions shared by every entry point:
 *   - Pointers named phi* are DEVICE pointers to the state, owned by the caller.  State
 *     layout: 1D [K][n]; 2D [ky][kx][n][n] with the x index fastest (node (i, j) of element
 *     (ex, ey) at offset ((ey*kx + ex)*n + j)*n + i); p-adaptive 2D meshes store element e
 *     (row-major over (ey, ex)) at offset off[e] with n_e*n_e values, off being the exclusive
 *     prefix sum of n_e^2.  SL_FP64 state is one double per node.  SL_MIXED state is
 *     double-float: a plane of sl_state_size floats "hi" at float offset 0 and a plane of as
 *     many floats "lo" at float offset P = sl_state_size rounded up to a multiple of 64 (so
 *     both planes start 256-byte aligned); the node value is hi + lo (about 48 significant
 *     bits).  sl_pack and sl_unpack convert from and to doubles.  A state buffer has
 *     sl_state_bytes bytes (8 per node, plus the padding of the mixed format) and starts on a
 *     16-byte boundary (state is moved with 16-byte vectors and bulk copies).
 *   - Pointers documented as "host" are host memory; everything else is device memory.
 *   - The library owns its tables, operators and workspace (allocated in sl_init and freed in
 *     sl_free).  All device work is enqueued on the stream given to sl_init; no call
 *     synchronises the stream except sl_mass, sl_energy, sl_sync and sl_run_host, which
 *     return host values.
 *   - Every function returns an sl_status.  Argument errors are reported before any work is
 *     enqueued and leave the state untouched; sl_last_error gives a one-line reason.  Errors
 *     found on the device (non-finite values, an energy iteration that hit its cap, a
 *     collocation solve that did not converge) are sticky bits read by sl_sync.  Nothing in
 *     the library aborts the process.
 */
#ifndef SL_H
#define SL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sl_ctx sl_ctx;

typedef enum {
  SL_OK = 0,
  SL_EINVAL = 1,       /* bad argument (null pointer, size, enum value)                  */
  SL_ENOMEM = 2,       /* device allocation failed                                       */
  SL_ECUDA = 3,        /* a CUDA runtime call failed                                     */
  SL_ECFL = 4,         /* displacement over one step would exceed one element width      */
  SL_EDEVICE = 5,      /* device status bits are set (see sl_sync)                       */
  SL_EUNSUPPORTED = 6  /* valid request that this build does not implement               */
} sl_status;

/* Solution node families (Sec. 3, eq. gaussquad): Gauss-Legendre, or Chebyshev-Gauss
 * xi_i = (1 - cos((i + 1/2) pi / n)) / 2.  Quadrature weights (eq. quad) are the Gauss
 * weights, or for Chebyshev-Gauss nodes the interpolatory (Fejer first-rule) weights. */
enum { SL_GAUSS_LEGENDRE = 0, SL_CHEB_GAUSS = 1 };

/* Arithmetic: SL_FP64 computes every step in double precision on double state.
 * SL_MIXED keeps double-float state and does the bulk arithmetic in float on increments
 * relative to a per-element reference value (so float rounding scales with the variation
 * inside an element), writing results back exactly.  In 1D it requires a constant velocity:
 * the whole linear step is then one operator shared by all elements. */
enum { SL_FP64 = 0, SL_MIXED = 1 };

/* Domain faces: periodic wrap, or an inflow face that sees the constant ghost value
 * (Sec. 4.3: boundary conditions through a specified ghost solution). */
enum { SL_BC_PERIODIC = 0, SL_BC_INFLOW = 1 };

/* Prescribed velocity fields (Sec. 4.2: velocity taken as prescribed).
 *   SL_VEL_CONST    p = {a, b}: constant (Sec. 5.1, 5.3)
 *   SL_VEL_ROTATION p = {omega, cx, cy}: u = -omega (y - cy), v = omega (x - cx)
 *   SL_VEL_SWIRL    p = {T}: u = sin^2(pi x) sin(2 pi y) cos(pi t / T),
 *                            v = -sin^2(pi y) sin(2 pi x) cos(pi t / T)
 *   SL_VEL_SINX     u = -sin x, 1D only (Sec. 5.2, eq. usin_lagr)
 *   SL_VEL_NODAL    a velocity given at the solution nodes, as an Eulerian solver on the same
 *                   elements provides it (Sec. 4.2: the particles start at the Gauss nodes, where
 *                   that velocity is known).  nodal points to DEVICE doubles laid out
 *                   [2][dim][state values]: the u (then, in 2D, v) node values at t and at t + dt
 *                   of the step, each in the context's state layout.  Between nodes the field is
 *                   the Lagrange interpolant of the element that contains the point (extrapolated
 *                   from the boundary element beyond a non-periodic face, wrapped across a
 *                   periodic one), linear in time over the step; on a face (within 1e-12 of
 *                   |x0| + |x1|, resp. |y0| + |y1|) it is the average over the elements sharing
 *                   it, so both sides see one velocity; div u comes from the same interpolants
 *                   and enters the value equation (eq. 4.8).  p = {umax, vmax}: bounds of |u| and
 *                   |v| that the caller supplies for sl_max_dt and the CFL check (the library
 *                   does not read the device array on the host).  Step k of sl_run reads the
 *                   array at nodal + k * nodal_step doubles (0: the same field every step).
 *                   FP64 contexts with one node count (no batch); other contexts return
 *                   SL_EUNSUPPORTED.  The caller keeps the array alive and unchanged while steps
 *                   that read it are in flight. */
enum { SL_VEL_CONST = 0, SL_VEL_ROTATION = 1, SL_VEL_SWIRL = 2, SL_VEL_SINX = 3, SL_VEL_NODAL = 4 };

/* Constraint rows of the least-squares fit (eq. matrix_a). */
enum { SL_C_BOUNDARY = 1, SL_C_MASS = 2, SL_C_ENERGY = 4 };

/* Fit: SL_FIT_HARD solves the lexicographic least-squares problem (constraints first, in the
 * least-squares sense, then nearest to the remapped values); SL_FIT_SOFT solves the paper's
 * stacked over-determined system (eq. matrix_a) by ordinary least squares. */
enum { SL_FIT_HARD = 0, SL_FIT_SOFT = 1 };

/* Interface values: SL_BV_INTERP evaluates the advected polynomial at the face
 * (eq. remap_bnd); SL_BV_BACKTRACK evaluates phi^n at the backward foot (eq. 4.11). */
enum { SL_BV_INTERP = 0, SL_BV_BACKTRACK = 1 };

/* Time-step rules for sl_max_dt (eq. 1d_delt_condition, 2d_delt_condition): half the minimum
 * spacing between adjacent nodes; the paper's step (the gap from the element edge to its first
 * node, factor 1: no particle leaves its element); half the paper's step.  Measured on the 2D
 * deforming flows (swirl, solid-body rotation with inflow walls) at fine meshes and n >= 8, the
 * paper's step sits at the stability limit: perturbations grow without bound (both precisions,
 * every constraint set, fit and interface rule), where half of it stays bounded. */
enum { SL_RULE_HALF_MIN_SPACING = 0, SL_RULE_PAPER = 1, SL_RULE_HALF_PAPER = 2 };

/* Sticky device status bits (sl_sync). */
enum {
  SL_ST_NONFINITE = 1u,      /* a non-finite value was written                          */
  SL_ST_PICARD_NOCONV = 2u,  /* the energy iteration hit its cap or was infeasible      */
  SL_ST_SOLVE_NOCONV = 4u,   /* the 2D collocation iteration did not reach its tolerance
                                (nor an accepted floor): the element keeps its best iterate */
  SL_ST_TIMEOUT = 8u,        /* a bounded wait for an asynchronous copy gave up (the step
                                left its output incomplete)                             */
  SL_ST_SOLVE_FLOOR = 16u    /* SL_MIXED 2D: a collocation solve that stalled or diverged
                                was accepted at a residual between the float floor (4e-6)
                                and 1e-4, relative to the largest collocation datum      */
};

typedef struct {
  int dim;               /* 1 or 2                                                          */
  int kx, ky;            /* elements per direction (ky = 1 in 1D)                           */
  double x0, x1, y0, y1; /* domain box (y0, y1 ignored in 1D)                               */
  int bc[4];             /* faces W, E, S, N (1D uses W, E)                                 */
  double ghost;          /* value at inflow domain faces                                    */
  const int32_t* order;  /* host, nullable: per-element node counts, [ky][kx] (p-adaptive) */
} sl_mesh;

typedef struct {
  int kind;              /* SL_VEL_*                                                        */
  double p[6];           /* parameters, see SL_VEL_*                                        */
  const double* nodal;   /* SL_VEL_NODAL: device node velocities (else ignored, may be NULL) */
  int64_t nodal_step;    /* SL_VEL_NODAL: doubles between the arrays of successive sl_run steps */
} sl_velocity;

typedef struct {
  unsigned constraints;  /* SL_C_* bits                                                     */
  int rk_order;          /* 1 (Euler), 2 (Heun), 3 (Kutta), 4 (classical)                   */
  int fit;               /* SL_FIT_HARD or SL_FIT_SOFT                                      */
  int bvalue;            /* SL_BV_INTERP or SL_BV_BACKTRACK                                 */
  double picard_rtol;    /* energy iteration stops when max|change| < rtol * max|phihat|;
                            0 selects 1e-13                                                 */
  int picard_cap;        /* iteration cap, 0 selects 60                                     */
} sl_options;

/* Create a context for one mesh.  n = nodes per direction (polynomial degree n - 1),
 * 2 <= n <= 17 (ignored when mesh->order is given, whose entries must lie in [2, 17]).
 * mesh->order makes a p-adaptive 2D mesh (1D: SL_EUNSUPPORTED): element (ex, ey) has
 * order[ey*kx + ex] nodes per direction, its state is stored at the CSR offset described
 * above, and a face between elements of different node counts is handled as follows: the
 * upwind value at a face point is the neighbour's remapped polynomial evaluated there, and the
 * mass/energy flux through the face is integrated once with the Gauss rule of the side with
 * more nodes, so both elements see the same flux and global mass telescopes.
 * cuda_stream: a cudaStream_t (0 = legacy default stream).  Precomputes, in host double
 * and long double arithmetic, the nodes, weights, face basis values and fit operators
 * (Sec. 3, eq. 3.5, quad, matrix_a) and uploads them.  On success *out owns device memory
 * until sl_free. */
sl_status sl_init(const sl_mesh* mesh, int n, int basis, int precision, void* cuda_stream,
                  sl_ctx** out);

/* Release a context and its device memory.  Null is ignored. */
void sl_free(sl_ctx* ctx);

/* Advance the state by one step from time t to t + dt (Sec. 4, steps a-d).  phi_in and
 * phi_out are distinct device buffers of sl_state_bytes bytes in the context's state format;
 * phi_in is only read.  Returns SL_ECFL when |u|max dt exceeds the element width, and
 * SL_EUNSUPPORTED for a combination this build does not implement (nothing is enqueued). */
sl_status sl_step(sl_ctx* ctx, const void* phi_in, void* phi_out, const sl_velocity* vel,
                  double t, double dt, const sl_options* opt);

/* Advance nsteps steps from t0 with a fixed dt (Sec. 4 per step), alternating between two
 * distinct device state buffers: phi_a holds the initial state; the result is in phi_a when
 * nsteps is even and in phi_b when it is odd (the other buffer holds the previous step).  The
 * steps are captured once into a CUDA graph on a stream owned by the context and replayed by
 * later calls with identical arguments (velocity, t0, dt, nsteps, options, buffers); the graph
 * is ordered after the work already enqueued on the context's stream, and that stream waits
 * for it.  Operators are prepared before the capture, so no host-to-device copy is recorded.
 * A batch runs every problem with the same t0 and dt (see sl_batch_create).  Argument and CFL
 * errors are reported before anything is enqueued; device errors are sticky bits (sl_sync). */
sl_status sl_run(sl_ctx* ctx, void* phi_a, void* phi_b, const sl_velocity* vel, double t0, double dt,
                 int nsteps, const sl_options* opt);

/* Time-dependent inflow (Dirichlet) data for the domain faces of a 1D FP64 context (Sec. 5.1,
 * the Dirichlet-versus-periodic comparison: the exact solution prescribed at the inflow; Sec. 4.3,
 * boundary conditions through a specified ghost solution).  values is a DEVICE array of doubles
 * owned by the caller, which must keep it alive and unchanged while steps that read it are in
 * flight; NULL returns to the mesh's constant ghost.  One record per step, of SL_INFLOW_RECORD
 * doubles: record[side * 5 + 0] is the ghost value at face `side` (0: x = x0, 1: x = x1) at
 * t + dt, where it enters the upwind value of eq. 4.12a; record[side * 5 + 1 + s] is the value
 * at t + c_s dt, the time of RK stage s (s < rk_order), where it enters the inflow flux of the
 * mass and energy targets (eq. remap_mass, remap_energy).  Only inflow faces (SL_BC_INFLOW on
 * that side) read it.  sl_step reads record 0; step k of sl_run reads the record at
 * values + k * step_stride (step_stride >= SL_INFLOW_RECORD when nsteps > 1; a graph recorded by
 * sl_run keeps the pointer it was recorded with).  Errors: SL_EINVAL for a negative stride,
 * SL_EUNSUPPORTED for a 2D, mixed-precision or batch context (nothing is changed). */
#define SL_INFLOW_RECORD 10
sl_status sl_set_inflow(sl_ctx* ctx, const double* values, int64_t step_stride);

/* Advance nsteps steps from t0 with a fixed dt, starting from and ending in HOST buffers of
 * sl_state_size doubles (node values in state layout, whatever the precision): copies host_in
 * to the device (converting to the state format), steps, converts back and copies the result
 * to host_out, then synchronises.  host_in and host_out may alias.  The device buffers this
 * needs are allocated on the first call and kept until sl_free. */
sl_status sl_run_host(sl_ctx* ctx, const double* host_in, double* host_out, const sl_velocity* vel,
                      double t0, double dt, int nsteps, const sl_options* opt);

/* Batches of independent 2D problems advanced by the same launches (one pair of kernel launches
 * per node count present, whatever the number of problems).  sl_batch_create builds a batch
 * context from nprob problem contexts (host array, 1 <= nprob <= 65535; each made by sl_init,
 * all with the same basis and precision, uniform or p-adaptive).  The batch state is the
 * problems' states concatenated in problem order, as one state of sl_state_size values in the
 * context's state format: problem p's node values start at value offset sl_batch_offset(batch,
 * p) (sl_batch_offset(batch, nprob) is the total; -1 on a bad argument).  For SL_MIXED the
 * planes span the whole batch, so a problem's part is reached through sl_unpack.  The batch
 * context works with every entry point taking a context; it keeps copies of the problems'
 * meshes (the problem contexts may be freed), uses the stream of probs[0], and is released with
 * sl_free.  sl_step advances every problem with the same t and dt; sl_batch_step takes host
 * arrays of nprob times and steps (each checked against its problem's element size, SL_ECFL).
 * sl_max_dt returns the smallest limit over the problems.  sl_mass and sl_energy sum over all
 * problems. */
sl_status sl_batch_create(int nprob, sl_ctx* const* probs, sl_ctx** batch);
sl_status sl_batch_step(sl_ctx* batch, const void* phi_in, void* phi_out, const sl_velocity* vel,
                        const double* t, const double* dt, const sl_options* opt);
int64_t sl_batch_offset(const sl_ctx* batch, int p);

/* Convert sl_state_size doubles (device) into the context's state format (device, sl_state_bytes
 * bytes), and back.  For SL_FP64 these are plain copies.  Enqueued on the context's stream. */
sl_status sl_pack(sl_ctx* ctx, const double* src, void* dst);
sl_status sl_unpack(sl_ctx* ctx, const void* src, double* dst);

/* Global mass sum_k integral phi and energy sum_k integral phi^2 (eq. quad summed over the
 * elements, diagnostics of Sec. 5), accumulated in double in a fixed order (deterministic).
 * *total is a host double; the call synchronises the stream. */
sl_status sl_mass(sl_ctx* ctx, const void* phi, double* total);
sl_status sl_energy(sl_ctx* ctx, const void* phi, double* total);

/* Synchronise the stream, return and clear the sticky device status bits (SL_ST_*). */
sl_status sl_sync(sl_ctx* ctx, uint32_t* status_bits);

/* Largest dt allowed by a time-step rule for this mesh and velocity (host computation). */
sl_status sl_max_dt(const sl_ctx* ctx, const sl_velocity* vel, int rule, double* dt);

/* Number of node values of the state, and bytes of one state buffer (-1 for a null ctx). */
int64_t sl_state_size(const sl_ctx* ctx);
int64_t sl_state_bytes(const sl_ctx* ctx);

/* Physical node coordinates in state layout, written to host arrays of sl_state_size
 * doubles (y may be null in 1D), for setting up initial data (a batch: every problem's nodes in
 * its own box). */
sl_status sl_node_coords(const sl_ctx* ctx, double* x, double* y);

/* Quadrature nodes and weights on [0, 1] of the context's basis for n nodes (host arrays). */
sl_status sl_nodes_weights(const sl_ctx* ctx, int n, double* xi, double* w);

/* Global integral sum_k h^d sum w (x) w phi^power of a double state, like sl_mass (power 1) and
 * sl_energy (power 2), for callers that cannot allocate device memory when they need it: code
 * that runs while a stream is being captured into a CUDA graph in global capture mode (where
 * cudaMalloc is not permitted), host loops under a hard latency budget (cudaMalloc may
 * synchronise the whole device), or applications whose memory pool owns all device memory.
 * The paper has no counterpart; this is a service of the library.
 *
 * It allocates nothing and needs no context.  Inputs: phi (device) holds nelem elements of
 * nper nodes (dim = 1) or nper x nper nodes (dim = 2) in state layout; w_host (host) holds the
 * nper quadrature weights on [0, 1] (sl_nodes_weights); scale is h (1D) or hx*hy (2D).  Output:
 * *total (device double) receives the integral.  Work is enqueued on cuda_stream; the call
 * does not synchronise.  The sum is deterministic (fixed order), but ordered differently from
 * sl_mass, so the two agree to rounding.
 *
 * Scratch: per-tile partial sums live in a fixed array of 65536 doubles (512 KB) in the
 * library's device memory, which every GPU that loads the library holds until the process
 * exits.  Inputs of more than SL_NOALLOC_MAX_VALUES values are rejected with SL_EINVAL (message
 * in sl_last_error(NULL)).  Every call shares that array: calls whose work overlaps on the GPU
 * (other streams, other host threads) race and must be serialised by the caller.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture begins.  Returns SL_ECUDA if
 * the lookup or a launch fails. */
#define SL_NOALLOC_MAX_VALUES ((int64_t)1 << 28)
sl_status sl_integral_noalloc(const double* phi, int64_t nelem, int nper, int dim, const double* w_host,
                              int power, double scale, double* total, void* cuda_stream);

/* Work counters of the two-dimensional SL_MIXED step for non-constant velocities, p-adaptive meshes
 * and batches (the kernels that solve the collocation system of eq. 5.4 per element), summed on the
 * device over every step since the last call:
 *   SL_CNT_ELEMS           element updates;
 *   SL_CNT_SOLVE_ITERS     residual evaluations of the collocation iteration (per element: the
 *                          iterations taken, including the one that met the tolerance);
 *   SL_CNT_SOLVE_FLOOR     solves accepted above the float floor (SL_ST_SOLVE_FLOOR);
 *   SL_CNT_SOLVE_NOCONV    solves not accepted (SL_ST_SOLVE_NOCONV);
 *   SL_CNT_ENERGY_APPLIED  elements whose linear fit missed the energy target, so that the energy
 *                          iteration of Sec. 4.3 ran;
 *   SL_CNT_PICARD_ITERS    iterations of that energy iteration;
 *   SL_CNT_PICARD_NOCONV   elements where it did not converge and the linear-constraint fit was
 *                          kept (SL_ST_PICARD_NOCONV);
 *   SL_CNT_FEET            outflow face points (per distinct RK stage time after t^n) whose
 *                          backward characteristic foot was traced for the mass/energy flux.
 * counts (host) receives SL_NCOUNTERS values; the call synchronises the context's stream and resets
 * the counters.  Other paths leave them unchanged. */
enum {
  SL_CNT_ELEMS = 0,
  SL_CNT_SOLVE_ITERS = 1,
  SL_CNT_SOLVE_FLOOR = 2,
  SL_CNT_SOLVE_NOCONV = 3,
  SL_CNT_ENERGY_APPLIED = 4,
  SL_CNT_PICARD_ITERS = 5,
  SL_CNT_PICARD_NOCONV = 6,
  SL_CNT_FEET = 7,
  SL_NCOUNTERS = 8
};
sl_status sl_counters(sl_ctx* ctx, uint64_t* counts);

/* Device time of the step's kernels, measured with CUDA events on the context's stream (the
 * stream the kernels are launched on).  sl_timing(ctx, 1) starts a session: every following sl_step,
 * sl_batch_step or sl_run_host step records an event before its first kernel, one between the two
 * phases of the two-dimensional general path (phase 1: advection, collocation solve, traces and face
 * outflow; phase 2: interface values, targets, fit and write-back) and one after its last kernel;
 * steps inside sl_run's captured graphs are not timed.  sl_timing(ctx, 0) ends the session and
 * releases its events.  Both synchronise the stream.  sl_timing_read synchronises and returns, for
 * the steps of the session so far, the summed milliseconds ms[0] of phase 1 (the whole kernel of a
 * single-kernel path), ms[1] of phase 2 (0 there) and ms[2] of both, and *nsteps, the number of timed
 * steps.  Timing adds three event records per step and nothing else to the work. */
sl_status sl_timing(sl_ctx* ctx, int enable);
sl_status sl_timing_read(sl_ctx* ctx, double* ms, int* nsteps);

/* Autotuner of the launch shapes of the kernels a step of this context runs with these
 * arguments.  The 2D shared-operator path (uniform mesh, constant velocity, mixed precision) has
 * a few compiled tile shapes (elements per CTA) per node count; the 2D general mixed path runs
 * persistent grids whose resident CTAs per SM can be held below the occupancy limit, per phase.
 * sl_tune times each candidate with CUDA events on the context's stream (one warm-up and three
 * timed steps from phi_in to phi_out; phi_in is only read, phi_out is overwritten), keeps the
 * fastest in the context, and records it under a key naming the device, the path, the mesh, the
 * node count and the options in the JSON file cache_path (a flat object of string keys and string
 * values, rewritten through a temporary file; null: no cache).  A key already in the file is
 * applied without timing.  Other paths have nothing to tune (no timing, default shapes).  Every
 * shape computes each element with the same arithmetic, so results do not depend on the choice.
 * choice (host, nullable, 4 ints): the tile index, the CTAs per SM of phase 1 and of phase 2
 * (0: the occupancy limit), and 1 if the choice came from the cache.  Synchronises the stream.
 * Errors: those of sl_step; SL_EINVAL for an unreadable or unwritable cache (nothing applied). */
sl_status sl_tune(sl_ctx* ctx, const void* phi_in, void* phi_out, const sl_velocity* vel, double t, double dt,
                  const sl_options* opt, const char* cache_path, int* choice);

/* Last error message of the context (or of the last failed sl_init when ctx is null). */
const char* sl_last_error(const sl_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SL_H */
