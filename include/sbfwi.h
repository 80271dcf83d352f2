/*
 * sbfwi.h -- C ABI of the GB300 library for the time-domain SBFEM full-waveform
 * inversion hot path (forward solve, misfit, time-reversed adjoint and the
 * velocity part of the Frechet kernel) of "Full-waveform inversion via the
 * scaled boundary finite element method" (arXiv 2501.06748).
 *
 * Conventions for every call
 * --------------------------
 *  - Return value: SBFWI_OK (0) or a negative SBFWI_E* code.  The message of the
 *    last failure on the calling thread is returned by sbfwi_last_error().
 *  - Floating-point data are IEEE binary64, C-contiguous.  Integer ids are int64.
 *  - Arrays are owned by the caller.  Handles (mesh, model, forward state) are
 *    owned by the library and released with the matching sbfwi_destroy_* call.
 *    A handle must not be used by two threads at once.
 *  - `mem` tells where the floating-point arrays named in a call's description
 *    live: SBFWI_MEM_HOST (ordinary or pinned host memory; the library stages
 *    them through the device) or SBFWI_MEM_DEVICE (device memory of the current
 *    CUDA device).  Id arrays (node ids) are always host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All device work of a call is ordered on it; calls return after the work is
 *    complete (host outputs are written, device outputs are ready).
 *  - Nothing here falls back to the CPU: without a usable CUDA device the
 *    compute calls return SBFWI_ECUDA.
 *
 * Nodal points (the parameters and the gradient live on them; Section 4 of the
 * paper defines the density "at the nodal points" and uses the solution fields
 * there directly):
 *    interior point (e, i, j), element e, radial point i = 0..N_r-2, boundary
 *    node j of the element (local numbering below), has index
 *        e*(N_r-1)*n_b + i*n_b + j
 *    and global boundary node g (radial point i = N_r-1, shared by the elements
 *    meeting there) has index n_int + g, n_int = n_elem*(N_r-1)*n_b.
 *    Its location is x0 + xi_i (x_j - x0) (Eq. (transformation)).
 *  Local numbering of an element's boundary nodes: order of first appearance
 *  when walking its line elements in the given (counter-clockwise) order.
 */
#ifndef SBFWI_H
#define SBFWI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SBFWI_OK = 0,
  SBFWI_EINVAL = -1,       /* bad argument or malformed mesh */
  SBFWI_ENOMEM = -2,       /* device or host allocation failed */
  SBFWI_ECUDA = -3,        /* CUDA runtime error (message has the CUDA text) */
  SBFWI_ETIMEOUT = -4,     /* a bounded device wait gave up */
  SBFWI_ESTATE = -5,       /* handle used in the wrong state */
  SBFWI_ESINGULAR = -6,    /* a pivot block or the global matrix is singular */
  SBFWI_EUNSUPPORTED = -7  /* valid request outside what this build implements */
};
enum { SBFWI_MEM_HOST = 0, SBFWI_MEM_DEVICE = 1 };
enum { SBFWI_RHO_GRID = 0, SBFWI_RHO_NODAL = 1 };
enum { SBFWI_GRAD_KERNEL = 0, SBFWI_GRAD_EXACT = 1 };
/* or-ed into the mode of sbfwi_adjoint_gradient: add into grad instead of overwriting */
enum { SBFWI_GRAD_ACCUMULATE = 0x100 };
/* sbfwi_forward's ckpt_every: choose the checkpoint interval automatically */
enum { SBFWI_CKPT_AUTO = -1 };

typedef struct sbfwi_mesh sbfwi_mesh;
typedef struct sbfwi_model sbfwi_model;
typedef struct sbfwi_fwdstate sbfwi_fwdstate;

/* Message of the last failure on this thread ("" if none).  Owned by the library. */
const char* sbfwi_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int sbfwi_version(void);

/*
 * sbfwi_build_mesh -- a mesh of 2-D scaled-boundary elements (Section 3: a
 * star-convex polygon per element, boundary discretised by line elements of
 * Lagrange order p, scaling centre (x0, y0), coordinate map
 * x = x0 + xi (x_b(eta) - x0), Eq. (transformation)).
 *
 *   node_xy     [n_nodes][2]   node coordinates
 *   elem_ptr    [n_elem+1]     element e owns line elements elem_ptr[e]..elem_ptr[e+1]-1
 *   line_nodes  [n_lines][p+1] global node ids of each line element, in the direction
 *                              of travel; an element's lines form a closed
 *                              counter-clockwise loop (end of one = start of next)
 *   centre_xy   [n_elem][2]    scaling centres
 *   p           line order, 1..8 (nodes equally spaced along straight lines)
 *   n_r         radial finite-difference points per element, N_r >= 3
 *               (xi_i = xi0 + i h, h = (1-xi0)/(N_r-1), Section 3.3)
 *   xi0         scaling-centre offset (the paper uses 1e-3)
 *
 * Checks: ids in range, closed CCW loops, straight lines with equally spaced
 * nodes, det J_b > 0 (scaling centre sees every line from its left).  Returns
 * SBFWI_EINVAL with the offending element in the message.  Elements may have
 * different numbers of line elements, hence of boundary nodes n_b(e) = p L(e)
 * (quadtree meshes whose sides are split at hanging vertices, polygons); at most
 * 40 per element (SBFWI_EUNSUPPORTED beyond).  The library pads every element to
 * the mesh's largest n_b internally; the nodal points seen by callers (nodal
 * densities and gradients) are unpadded: the N_r - 1 interior radial points of
 * each element's n_b(e) rays in element order, radial index major, then the
 * global nodes.  All arrays are host memory, copied.
 */
int sbfwi_build_mesh(sbfwi_mesh** out, const double* node_xy, int64_t n_nodes,
                     const int64_t* elem_ptr, const int64_t* line_nodes, int64_t n_lines,
                     const double* centre_xy, int64_t n_elem, int32_t p, int32_t n_r, double xi0);

/*
 * sbfwi_build_mesh3d -- a mesh of 3-D scaled-boundary elements: the paper's Section 3
 * preamble says a three-dimensional formulation needs only minor changes; this build
 * carries it out for a boundary surface.  Each element is a star-convex polyhedron
 * whose boundary is a set of quadrilateral faces of Lagrange order p, with scaling
 * centre x0 and the map x = x0 + xi (x_b(eta, zeta) - x0).  The coefficient matrices
 * are the surface integrals E0 = int rho c^2 N^T (b1.b1) N det J_b, E1 = int rho c^2
 * B2^T b1 N det J_b, E2 = int rho c^2 B2^T B2 det J_b, M0 = int rho N^T N det J_b with
 * B2 = b2 N_eta + b3 N_zeta and b1, b2, b3 the columns of the inverse boundary Jacobian
 * (rows x_b - x0, x_b,eta, x_b,zeta); the radial equation is
 *   xi^2 E0 u'' + xi (2 E0 + E1^T - E1 + xi E0') u' + (E1^T - E2 + xi E1^T') u - xi^2 M0 u_tt = 0
 * (the 2-D equation with 2 E0 for E0 in the u' coefficient and + E1^T in the u
 * coefficient), discretised, condensed and stepped exactly as in 2-D.
 *
 *   node_xyz    [n_nodes][3]         node coordinates
 *   elem_ptr    [n_elem+1]           element e owns faces elem_ptr[e]..elem_ptr[e+1]-1
 *   face_nodes  [n_faces][(p+1)^2]   global node ids of each face in tensor order: node
 *                                    (a, b) at a + (p+1) b, a along the face's first
 *                                    direction eta, b along zeta, with eta x zeta
 *                                    pointing out of the element
 *   centre_xyz  [n_elem][3]          scaling centres
 *   p           face order, 1..4 (nodes equally spaced on the bilinear patch of the
 *               face's corners; planar faces give exact quadrature)
 *   n_r, xi0    as sbfwi_build_mesh
 *
 * Checks: ids in range, at least four faces per element, nodes on the bilinear patch of
 * the corners, det J_b > 0 at the corners and middle of every face, every face edge
 * shared by exactly two faces of the element (a closed surface).  Returns
 * SBFWI_EINVAL with the offending element in the message, SBFWI_EUNSUPPORTED beyond 40
 * boundary nodes per element (a hexahedron has 8 at p = 1 and 26 at p = 2).  The nodal
 * points and their order are those of the 2-D meshes.  A 3-D mesh takes its model from
 * sbfwi_set_model3d; the comparison method, the full kernel's gradient term and the
 * exact adjoint are not built for it (SBFWI_EINVAL / SBFWI_EUNSUPPORTED).  All arrays
 * are host memory, copied.
 */
int sbfwi_build_mesh3d(sbfwi_mesh** out, const double* node_xyz, int64_t n_nodes,
                       const int64_t* elem_ptr, const int64_t* face_nodes, int64_t n_faces,
                       const double* centre_xyz, int64_t n_elem, int32_t p, int32_t n_r, double xi0);

/* info[0..7] = n_elem, n_nodes, n_b (the largest), N_r, n_nodal (= n_int + n_nodes),
 * n_int (= (N_r - 1) x the sum of n_b(e)), levels of the global elimination tree,
 * nonzeros kept by the global factors. */
int sbfwi_mesh_info(const sbfwi_mesh* mesh, int64_t* info);
void sbfwi_destroy_mesh(sbfwi_mesh* mesh);

/*
 * sbfwi_set_model -- set-up of the path for one density model and time step
 * (per model, not per step; Section 3):
 *   density on the nodal points; coefficient matrices E0, E1, E2, M0 at every
 *   radial point (Eq. (Es)); radial derivatives of E0, E1; blocks of
 *   Eq. (system); condensation (pivots, Thomas sweep, last-row elimination and
 *   2x2 closure giving the element dynamic stiffness S and the effective-source
 *   operator); assembly and factorisation of the global boundary matrix sum_e S_e.
 *   The set-up runs in double-double arithmetic and rounds its results to FP64.
 *
 *   c        wave speed (constant, Section 3)
 *   rho      SBFWI_RHO_GRID:  [gy][gx] cell-centred values on [0,lx]x[0,ly],
 *                             mapped to nodal points by bilinear interpolation
 *                             (clamped at the edges);
 *            SBFWI_RHO_NODAL: [n_nodal] values on the nodal points (gx, gy, lx, ly unused).
 *            All values must be > 0 (SBFWI_EINVAL).
 *   dt, beta, gamma  Newmark parameters (Eq. (Newmark)); beta > 0.
 *   mem      where rho lives.
 * Errors: SBFWI_ESINGULAR if a pivot block or a separator block of the global
 * matrix cannot be inverted.  The model keeps a reference to `mesh`, which must
 * outlive it.
 */
int sbfwi_set_model(sbfwi_model** out, const sbfwi_mesh* mesh, double c, const double* rho,
                    int rho_kind, int64_t gx, int64_t gy, double lx, double ly,
                    double dt, double beta, double gamma, int mem, void* stream);
void sbfwi_destroy_model(sbfwi_model* model);

/*
 * sbfwi_set_model3d -- sbfwi_set_model for a mesh from sbfwi_build_mesh3d.
 *   rho  SBFWI_RHO_GRID:  [gz][gy][gx] cell-centred values on [0,lx]x[0,ly]x[0,lz],
 *                         mapped to nodal points by trilinear interpolation (clamped at
 *                         the edges); the gradient comes back on the same grid;
 *        SBFWI_RHO_NODAL: [n_nodal] values on the nodal points.
 * Other arguments and errors as sbfwi_set_model; SBFWI_EINVAL for a 2-D mesh.
 */
int sbfwi_set_model3d(sbfwi_model** out, const sbfwi_mesh* mesh, double c, const double* rho,
                      int rho_kind, int64_t gx, int64_t gy, int64_t gz, double lx, double ly, double lz,
                      double dt, double beta, double gamma, int mem, void* stream);

/*
 * sbfwi_set_model_lfe -- the same set-up for the paper's comparison method, the
 * low-frequency expansion of the reduced equation (Section 3.2): the density is held
 * constant along every radial line (its value at the element's boundary node), each
 * element gets K (Riccati) and M (Lyapunov, sbfwi_lfe_element_matrices), and the global
 * system sum_e K_e + M_e / (beta dt^2) is factorised.  Forward and adjoint passes on
 * the model then step M u'' + K u = f with Newmark on the boundary nodes only (no radial
 * interior); the gradient lives on the boundary nodes (interior nodal points get zero).
 * Arguments and errors as sbfwi_set_model; SBFWI_ESINGULAR also when an element's
 * Riccati or Lyapunov solve fails.  The full kernel (sbfwi_set_kernel_terms) does not
 * apply (SBFWI_EUNSUPPORTED at the forward call).
 */
int sbfwi_set_model_lfe(sbfwi_model** out, const sbfwi_mesh* mesh, double c, const double* rho,
                        int rho_kind, int64_t gx, int64_t gy, double lx, double ly,
                        double dt, double beta, double gamma, int mem, void* stream);

/*
 * sbfwi_set_schedule -- how the time loops of later sbfwi_forward and
 * sbfwi_adjoint_gradient calls on `model` run.  Not part of the paper: a
 * performance choice between kernels that compute the same method (results agree
 * within rounding, ~1e-13 relative on traces).  An autotuner times the candidates
 * and keeps the fastest (paper_2501_06748_gb300/autotune.py).
 *
 *   element  SBFWI_ELEMENT_AUTO: the tensor-core element kernel for a padded n_b of
 *            at most 16 or 21..32 with at most 8 shots per pass, else FP64 (the
 *            SBFWI_ELEMENT=fp64 environment variable forces FP64);
 *            SBFWI_ELEMENT_TENSOR: the tensor-core kernel wherever one exists
 *            (padded n_b <= 32, <= 8 shots; SBFWI_EUNSUPPORTED at the time-loop
 *            call otherwise; its operator digits are prepared on first use);
 *            SBFWI_ELEMENT_FP64: the FP64 kernel.
 *            SBFWI_ELEMENT_MIXED: on a mesh whose elements have different n_b (padded
 *            beyond 16), the elements with n_b <= 16 on the one-tile tensor-core kernel
 *            and the others on the FP64 kernel, two launches per step over element lists
 *            (SBFWI_EUNSUPPORTED at the time-loop call unless both classes exist and at
 *            most 8 shots run); AUTO picks it for a padded n_b of 17..20 or beyond 32.
 *   solve    SBFWI_SOLVE_AUTO: the dataflow solve (SBFWI_SOLVE=barrier|levels in
 *            the environment selects the others); SBFWI_SOLVE_DATAFLOW: one
 *            cooperative launch, tasks ordered by dependencies; SBFWI_SOLVE_BARRIER:
 *            one cooperative launch, grid barriers between tree levels;
 *            SBFWI_SOLVE_LEVELS: one launch per tree level and direction.  The
 *            cooperative schedules need a device that launches cooperatively
 *            (SBFWI_EUNSUPPORTED at the time-loop call otherwise).
 *
 * A checkpointed forward state must be consumed by an adjoint with the same
 * element kernel (SBFWI_ESTATE otherwise).  Errors: SBFWI_EINVAL for a NULL model
 * or an unknown value.
 */
/*
 * sbfwi_lfe_element_matrices -- the element stiffness K and mass M of the paper's
 * comparison method, the low-frequency expansion of the reduced element equation
 * (Section 3.2: density constant along xi, S ~ K - omega^2 M): K from the Riccati
 * equation (K - E1) E0^-1 (K - E1^T) - E2 = 0 (the solution whose modes are bounded at
 * the scaling centre, with the constant mode), M from the Lyapunov equation
 * (K - E1) E0^-1 M + M E0^-1 (K - E1^T) + 2 M - M0 = 0.
 *   E0, E1, E2, M0  [n_b][n_b] host, row-major, the element's coefficient matrices
 *                   (Eq. (Es)) for its density along the boundary
 *   K, M            [n_b][n_b] host outputs
 * Host computation in FP64 (matrix sign function for the Riccati subspace, dense
 * solve for the Lyapunov equation); no device use.  Errors: SBFWI_EINVAL (NULL,
 * n_b outside 2..40), SBFWI_ESINGULAR (a singular E0 or a failed iteration).
 */
int sbfwi_lfe_element_matrices(const double* E0, const double* E1, const double* E2, const double* M0,
                               int32_t n_b, double* K, double* M);

/*
 * sbfwi_set_kernel_terms -- which terms of the Frechet kernel (Section 2:
 * K_rho = int d_t lambda d_t u - c^2 grad lambda . grad u dt) later adjoint gradients
 * on `model` accumulate.
 *   SBFWI_TERMS_VELOCITY (default): the velocity term only, as the paper does
 *     (Section 4).
 *   SBFWI_TERMS_FULL: both terms.  The gradient at a nodal point comes from the
 *     coordinate map of each element line through it (second-order differences along
 *     the radial grid, the line's Lagrange derivative along it; the mean over the
 *     element lines that meet at the point).  Forward passes then also keep the
 *     nodal displacements of every step (twice the stored field); with checkpoints
 *     (ckpt_every != 0) the adjoint's recompute windows keep them (twice the window).
 * Errors: SBFWI_EINVAL for a NULL model or an unknown value.
 */
enum { SBFWI_TERMS_VELOCITY = 0, SBFWI_TERMS_FULL = 1 };
int sbfwi_set_kernel_terms(sbfwi_model* model, int terms);

/*
 * sbfwi_set_gradient_mode -- which gradient later forward passes on `model` are kept for.
 *   SBFWI_GRAD_KERNEL (default): the paper's gradient (Section 2 adjoint equation run in
 *     reversed time, Section 4 velocity kernel); a stored forward field holds the nodal
 *     velocities of every step.
 *   SBFWI_GRAD_EXACT: the exact derivative of the discrete misfit E (Eq. (misfit)) with
 *     respect to the nodal densities, i.e. the adjoint/stationarity conditions of Section 2
 *     applied to the discrete system of Section 3.3 (Eq. (system) with its boundary-condition
 *     rows, the condensation and Eq. (Newmark)) instead of the continuous equation.  The
 *     radial finite-difference operator is not symmetric, so this differs from the paper's
 *     kernel; it is what finite differences of E measure.  Forward passes then run the FP64
 *     element kernel and a stored forward field holds the nodal displacements and
 *     accelerations of every step (twice the velocity store); checkpointed forward states
 *     serve both modes.  The first exact adjoint on a model prepares its extra operators
 *     (the inverses of the modified pivot blocks, per element ~(N_r + 5) n_b^2 doubles, and
 *     the transposed global factors).
 * Errors: SBFWI_EINVAL for a NULL model or an unknown mode; SBFWI_EUNSUPPORTED for a
 * comparison-method model (sbfwi_set_model_lfe), whose exact adjoint is not built.
 */
int sbfwi_set_gradient_mode(sbfwi_model* model, int mode);

enum { SBFWI_ELEMENT_AUTO = 0, SBFWI_ELEMENT_TENSOR = 1, SBFWI_ELEMENT_FP64 = 2, SBFWI_ELEMENT_MIXED = 3 };
enum { SBFWI_SOLVE_AUTO = 0, SBFWI_SOLVE_DATAFLOW = 1, SBFWI_SOLVE_BARRIER = 2, SBFWI_SOLVE_LEVELS = 3 };
int sbfwi_set_schedule(sbfwi_model* model, int element, int solve);

/*
 * sbfwi_forward -- forward solve of n_shots independent shots on the model
 * (Section 2, Eq. (main); zero initial state), K Newmark steps.  Each step:
 * residual sources (Eq. (ODE_Newmark)), forward condensation sweep and
 * effective source of every element, global boundary solve, radial
 * back-substitution and Newmark update (Section 3.3).
 *
 *   src_node    [n_shots]          host; node of shot s's point source
 *   src_wavelet [n_shots][K]       sample k is added to the boundary right-hand
 *                                  side at src_node[s] for the step that produces
 *                                  the state at t_{k+1} = (k+1) dt
 *   rec_node    [n_rec]            host; receiver nodes shared by all shots (distinct)
 *   traces      [n_shots][n_rec][K] out: u at the receivers at t_{k+1}
 *   keep        if not NULL, receives a forward state for sbfwi_adjoint_gradient.
 *   ckpt_every  what that state holds (ignored without keep):
 *               0   the nodal velocities of every step, as Section 4 stores the
 *                   forward field for the adjoint: K * n_nodal * n_shots * 8 bytes
 *                   of device memory;
 *               c>0 the complete Newmark state before steps c, 2c, ... only
 *                   (checkpoints); the adjoint recomputes the forward field one
 *                   window of c steps at a time from them (one more forward solve
 *                   in time, memory (ceil(K/c) - 1) checkpoints here plus
 *                   c * n_nodal * n_shots * 8 bytes during the adjoint);
 *               SBFWI_CKPT_AUTO (-1) picks the c that minimises that memory.
 *               The traces, and the gradient of the adjoint, are bit for bit the
 *               same for every ckpt_every.  SBFWI_ENOMEM if the state does not fit.
 *   mem         where src_wavelet and traces live.
 */
int sbfwi_forward(sbfwi_model* model, int32_t n_shots, const int64_t* src_node,
                  const double* src_wavelet, int32_t n_rec, const int64_t* rec_node, int64_t K,
                  double* traces, sbfwi_fwdstate** keep, int64_t ckpt_every, int mem, void* stream);

/*
 * sbfwi_misfit -- E = 1/2 sum_{shot,rec} int (d - u)^2 dt (Eq. (misfit)) with the
 * rectangle rule over the n trace samples: E = 0.5 * dt * sum (observed - traces)^2.
 *   traces, observed  [n]; residual_out [n] (nullable) receives observed - traces.
 *   E_out  host pointer.  mem applies to traces, observed, residual_out.
 */
int sbfwi_misfit(const double* traces, const double* observed, int64_t n, double dt,
                 double* E_out, double* residual_out, int mem, void* stream);

/*
 * sbfwi_misfit_noalloc -- the same misfit as sbfwi_misfit, for callers that cannot
 * let the library allocate device memory.  The paper has no counterpart; this is
 * a service of the library.  Typical callers: a framework that has already
 * reserved nearly all device memory in its own pool, a real-time loop that must
 * not enter the driver's allocator (cudaMalloc/cudaFree can block and
 * synchronise), or a process held to a fixed memory budget.
 *
 *   traces, observed [n], residual_out [n] (nullable), E_out [1]: all DEVICE
 *   pointers (SBFWI_EINVAL otherwise).  n <= 268435456 (4096 blocks of 65536
 *   samples); larger n is rejected with SBFWI_EINVAL before any work is queued.
 *
 * The per-block partial sums go to a fixed 32 KiB array compiled into the
 * library (held by every device that loads it until the process exits) instead
 * of a buffer allocated per call.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  The first call on a device looks up that array's
 * device address (once per device, with that device current); make that first
 * call before capturing a stream into a CUDA graph.  The work is only enqueued
 * on `stream`: E_out and residual_out are valid once the stream reaches it.
 * All calls share the array, so calls that may run at the same time on the GPU
 * (different streams without ordering between them) race and can return wrong
 * values; order them on one stream.  Every call overwrites the partial sums it
 * uses, so nothing from an earlier call leaks into a later one.
 */
int sbfwi_misfit_noalloc(const double* traces, const double* observed, int64_t n, double dt,
                         double* E_out, double* residual_out, void* stream);

/*
 * sbfwi_adjoint_gradient -- time-reversed adjoint solve and zero-lag
 * cross-correlation (Section 2: adjoint equation and Frechet kernel; Section 4:
 * the c^2 grad(lambda).grad(u) term is dropped and the nodal fields are used
 * directly).  Adjoint step m (0-based) injects residual[s][r][K-1-m] at
 * rec_node[r] (same sign slot as the forward source) and accumulates
 *     g(node) += dt * sum_s udot_fwd[K-1-m](node, s) * lambdadot^{m+1}(node, s).
 * With SBFWI_GRAD_EXACT instead: g = dE/drho of the discrete path, E = 0.5 dt sum
 * residual^2 (residual = d - u as from sbfwi_misfit), by the transposed condensation
 * and global solve run backwards in time; summed over shots (see sbfwi_set_gradient_mode).
 *
 *   fwdstate  from sbfwi_forward(..., keep, ...) on the same model; not consumed.
 *             If it holds checkpoints, the forward field is recomputed window by
 *             window (last window first) with the element kernel that wrote them
 *             (SBFWI_ESTATE if SBFWI_ELEMENT now selects the other one).
 *   residual  [n_shots][n_rec][K] (d - u, as from sbfwi_misfit)
 *   mode      SBFWI_GRAD_KERNEL (the paper's kernel) or SBFWI_GRAD_EXACT (the exact
 *             derivative; SBFWI_ESTATE unless the model was in SBFWI_GRAD_EXACT mode
 *             when the forward state was made; SBFWI_GRAD_KERNEL on a stored field kept
 *             for the exact adjoint is SBFWI_ESTATE too).  With SBFWI_GRAD_ACCUMULATE
 *             or-ed in, the result is added to grad (gradients of shot batches run one
 *             after the other).
 *   grad      out: [gy][gx] (model set with SBFWI_RHO_GRID, the transpose of the
 *             bilinear map) or [n_nodal] (SBFWI_RHO_NODAL).
 *   mem       where residual and grad live.
 */
int sbfwi_adjoint_gradient(sbfwi_model* model, sbfwi_fwdstate* fwdstate, const double* residual,
                           int mode, double* grad, int mem, void* stream);

/*
 * Sessions: continuous batching of shot requests on one model (a service of the library
 * for serving; the numerics are those of sbfwi_forward and sbfwi_adjoint_gradient with
 * the paper's kernel, Section 2 and Section 4).  A session is a time loop whose B shot
 * columns ("slots") carry independent requests.  It advances in windows of `window`
 * Newmark steps; between windows a request can be admitted into a free slot (its state
 * column is zeroed, so the slot starts its own step 0 at the next window) and a finished
 * one collected, while the other slots keep running.  Every request's result is the same
 * as that shot run alone through sbfwi_forward / sbfwi_adjoint_gradient (to rounding: the
 * element kernels treat the shot columns independently).
 *
 *   kind      SBFWI_SESSION_FORWARD: a request is one point source (src_node, wavelet
 *             values[K]); its result is the traces [n_rec][K] at the session's receivers;
 *             with `field` (device, [K][n_nodal] doubles, caller-owned) its nodal
 *             velocities of every step are written there for a later adjoint.
 *             SBFWI_SESSION_ADJOINT: a request is a residual values[n_rec][K] (d - u, as
 *             from sbfwi_misfit) with the forward velocities `field` of its shot (as
 *             written by a forward session); its result is the gradient of the paper's
 *             kernel for that shot on the model's parameter layout ([gy][gx] or [n_nodal]).
 *   slots     1..16 shot columns; window 1..100000 steps per sbfwi_session_step.
 *   rec_node  [n_rec] distinct receiver nodes (host), shared by the session's requests.
 *
 * sbfwi_session_step runs one window of every slot whose request is not finished and
 * reports in finished[slots] (nullable) which slots hold a finished, uncollected request.
 * sbfwi_session_collect copies a finished slot's result to `out` (mem) and frees the slot.
 * Calls are synchronous on `stream` (given at creation).  Errors: SBFWI_EINVAL (bad
 * argument), SBFWI_ESTATE (admission to a busy slot, collection of an unfinished one),
 * SBFWI_EUNSUPPORTED (a model set for the full kernel or the exact adjoint).  The model
 * must outlive the session; a session must not be used by two threads at once.
 */
enum { SBFWI_SESSION_FORWARD = 0, SBFWI_SESSION_ADJOINT = 1 };
typedef struct sbfwi_session sbfwi_session;
int sbfwi_session_create(sbfwi_session** out, sbfwi_model* model, int32_t kind, int32_t slots, int32_t n_rec,
                         const int64_t* rec_node, int32_t window, void* stream);
int sbfwi_session_admit(sbfwi_session* session, int32_t slot, int64_t src_node, const double* values, int64_t K,
                        double* field, int mem);
int sbfwi_session_step(sbfwi_session* session, int32_t* finished);
int sbfwi_session_collect(sbfwi_session* session, int32_t slot, double* out, int mem);
/* info[0..4] = doubles per step of a forward field (the rows of `field`), steps run so far,
 * slots, window, slots holding a request. */
int sbfwi_session_info(const sbfwi_session* session, int64_t* info);
void sbfwi_session_destroy(sbfwi_session* session);

/*
 * sbfwi_destroy_fwdstate -- frees a forward state.  Its velocity or checkpoint
 * store (the largest allocation of the library, K * n_nodal * n_shots * 8 bytes
 * for a stored field) is kept in a one-slot cache instead of being freed, and the
 * next sbfwi_forward on the same device whose store is at least as large and at
 * most a third larger reuses it (an evaluation loop then allocates it once).
 * sbfwi_release_cache() frees the cached store; a forward that needs a store that
 * the cached one does not fit frees the cached one first.  (A service of the
 * library; the paper has no counterpart.)
 */
void sbfwi_destroy_fwdstate(sbfwi_fwdstate* state);
int sbfwi_release_cache(void);

/*
 * Tracing of the library's kernels (process-wide, not thread-safe).
 * sbfwi_profile_enable(1) makes every later call record CUDA event pairs on its
 * stream around each phase: 0 = set-up kernels (one interval per
 * sbfwi_set_model), 1 = the fused element step kernel (one interval per launch),
 * 2 = the global boundary solve (one interval per time step: all tree levels,
 * both passes), 3 = everything else (boundary update, sources, misfit,
 * gradient reduction).  Launch counts are kept whether or not timing is on.
 * sbfwi_profile_read fills ms[4] (device milliseconds), intervals[4] and
 * launches[4] (all nullable) and, if reset != 0, clears the counters.
 */
int sbfwi_profile_enable(int on);
int sbfwi_profile_read(double* ms, int64_t* intervals, int64_t* launches, int reset);

/*
 * Per-level tracing of the one-launch global solve with grid barriers between
 * levels (SBFWI_SOLVE=barrier; a diagnostic of this implementation, the paper does
 * not specify the solver; the default dataflow solve has no levels to time).
 * While profiling is on, every such launch reads the global timer around each phase (a tree
 * level of one pass, between two grid barriers).  Phases 0..L-1 are the forward
 * (leaves -> root) levels, L..2L-1 the backward levels (root -> leaves).  Slots
 * [0, 2L): wall time of the phase seen by block 0 (the last phase ends when block
 * 0 finishes); [2L, 4L): the longest time one block spent in its tasks of the
 * phase (maximum over blocks and solves, not a mean); [4L, 6L): the time blocks
 * spent in their tasks of the phase, summed over blocks.  Fills us[min(cap, 6L)]
 * with microseconds per solve (per solve and block for the maxima as recorded),
 * *n_slots = 6L (0 if nothing was recorded), *steps = solves recorded; reset != 0
 * clears the accumulators.
 * Synchronises the current device.  SBFWI_ESTATE if the trace lives on another
 * device.
 */
int sbfwi_profile_solve_levels(double* us, int32_t cap, int32_t* n_slots, int64_t* steps, int reset);

/*
 * Per-phase tracing of the dataflow global solve (the default schedule; a diagnostic
 * of this implementation, the paper does not specify the solver).  While profiling is
 * on, every such launch stamps the global timer when a block starts, when it claims an
 * item, when the item's inputs are ready and when the item has finished (the last 64
 * solves are kept).  A phase is one tree level of one pass: phases 0..L-1 are the
 * forward levels (leaves -> root), L..2L-1 the backward levels (root -> leaves).  Fills
 * us[min(cap, 8L)] with, per phase: [0, 2L) the time from the solve's first block start
 * (the first of its launches: a solve whose upper levels need a large staging area runs as
 * three launches in stream order) to the phase's last item finishing (the phase's
 * completion time), [2L, 4L)
 * the mean execution time of an item (inputs ready -> finished), [4L, 6L) the mean
 * time an item waited for its inputs after being claimed, [6L, 8L) items per solve;
 * microseconds, averaged over the recorded solves.  *n_slots = 8L (0 if nothing was
 * recorded), *steps = solves recorded; reset != 0 starts a new record.  Synchronises
 * the current device.  SBFWI_ESTATE if the trace lives on another device.
 */
int sbfwi_profile_solve_flow(double* us, int32_t cap, int32_t* n_slots, int64_t* steps, int reset);

/*
 * Failure-detection self-test (no counterpart in the paper; a guard of this
 * implementation).  Every device-side wait of the library is bounded: the grid
 * barrier between the tree levels of the global solve gives up after a budget of
 * clock cycles, records SBFWI_ETIMEOUT in a device status word and returns, so a
 * block that never arrives turns into an error code, not a hung device.  This
 * call runs that same barrier `rounds` times in a cooperative launch of n_blocks
 * blocks (64 threads each) of which the last n_absent return without arriving.
 *   n_absent = 0   every barrier completes; returns SBFWI_OK.
 *   n_absent > 0   the first barrier times out after about budget_cycles SM
 *                  cycles; returns SBFWI_ETIMEOUT and the device stays usable.
 * Synchronous on `stream`.  SBFWI_EINVAL if n_blocks exceeds what can be
 * co-resident, n_absent is not in [0, n_blocks), budget_cycles is not in
 * [1e3, 4e9] or rounds is not in [1, 1000].
 */
int sbfwi_selftest_barrier(int32_t n_blocks, int32_t n_absent, int64_t budget_cycles, int32_t rounds, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SBFWI_H */
