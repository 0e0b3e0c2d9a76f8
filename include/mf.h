/*
 * mf.h -- C ABI of the GB300 (sm_103a) FEM assembly + Krylov library.
 *
 * The library builds the global sparse system K x = d of a linearised weak form
 * on a mesh and solves it, after MetaFEM (Xie, Ehmann, Cao, arXiv 2111.03541):
 * the problem statement of Sec. 1 fixes K x = d by the forms, the element type
 * and order, the quadrature and the dof numbering; Sec. 2.2 Block B builds the
 * dof and sparse-entry maps, Block D-2/D-3 accumulate the residual and the
 * tangent, Block D-4 solves.  Three hand-lowered forms are provided: thermal
 * conduction (Sec. 4.1), linear elasticity (Sec. 4.2) and the Picard-linearised
 * Navier-Stokes domain form on Taylor-Hood elements (Sec. 4.3).
 *
 * Conventions shared by every call:
 *  - Data pointers are DEVICE pointers owned by the caller unless stated.
 *    The library owns only its opaque handles and the arrays inside them,
 *    which the matching *_destroy call frees.
 *  - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream).  Errors found by kernels
 *    (non-finite coefficient, bad index) are latched in a device status word
 *    and returned by the next mf_sync_status() or mf_solve().
 *  - No call aborts, traps or prints.  Invalid arguments return
 *    MF_ERR_INVALID_ARG without launching anything; mf_last_error() gives a
 *    thread-local message for the last failure.
 *  - K is returned positive: the paper's tangent dd/dphi of the conduction
 *    and elasticity residuals carries the opposite sign; the flow form keeps
 *    the paper's signs.  All indices are 0-based.
 *  - Dof numbering (Block B-3): thermal dof = node; elasticity dof =
 *    3 node + c (node-interleaved); flow dofs [u1 (n_nodes) | u2 (n_nodes) |
 *    p (n_pnodes)] (variable-major as in Block B-3).
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MF_OK = 0,
    MF_ERR_INVALID_ARG = 1,  /* bad pointer, size or enum; nothing launched */
    MF_ERR_BAD_MESH = 2,     /* connectivity out of range, or detJ <= 0 at a point */
    MF_ERR_NONFINITE = 3,    /* NaN/Inf coefficient, coordinate or residual */
    MF_ERR_OOM = 4,          /* device allocation failed */
    MF_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    MF_ERR_NOT_CONVERGED = 6,/* iteration cap reached before the tolerance */
    MF_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
    MF_ERR_UNSUPPORTED = 8   /* combination not provided (e.g. node valence too high) */
} mf_status;

typedef enum { MF_P1_TRI = 0, MF_P2_TRI = 1, MF_Q1_HEX = 2, MF_Q2S_HEX = 3, MF_P2_TET = 4, MF_Q2S_QUAD = 5 } mf_elem;
typedef enum {
    MF_FORM_THERMAL = 0, MF_FORM_ELASTIC = 1, MF_FORM_OSEEN = 2, MF_FORM_CAPACITY = 3,
    MF_FORM_NS = 4  /* steady Navier-Stokes with SUPG, Newton tangent (Sec. 4.3) */
} mf_form;
typedef enum { MF_PREC_FP64 = 0, MF_PREC_MIXED = 1 } mf_prec;
typedef enum {
    MF_SOLVER_PCG = 0, MF_SOLVER_GMRES = 1, MF_SOLVER_PCG_REFINED = 2, MF_SOLVER_GMRES_FLOW_MG = 3
} mf_solver;

typedef struct mf_mesh mf_mesh;
typedef struct mf_pattern mf_pattern;
typedef struct mf_flow_mg mf_flow_mg;

/* Mesh description (Block B-1: elements and their element->control-point map).
 * coords [n_nodes][dim] f64 AoS; conn [n_elems][npe] int32 with npe = 3 (P1),
 * 6 (P2: vertices, then midpoints of edges (0,1), (1,2), (2,0)), 8 (Q1: node
 * a = i + 2j + 4k at reference corner (2i-1, 2j-1, 2k-1)), 20 (Q2S: the
 * 20-node serendipity brick of the paper's experiments; the 8 vertices as Q1,
 * then the edge midpoints: x edges 8 + j + 2k at (0, 2j-1, 2k-1), y edges
 * 12 + i + 2k, z edges 16 + i + 2j; edges straight, midpoints at the mean of
 * their ends, so the geometry is the vertices' trilinear map; thermal and
 * elasticity forms (Sec. 4.1, Sec. 4.2), FP64, 3 x 3 x 3 Gauss, up to 128
 * neighbours per node), 10 (P2T: the quadratic tetrahedron of the paper's 3D
 * experiments; vertices 0..3 positively oriented, then the midpoints of
 * edges (0,1), (1,2), (2,0), (0,3), (1,3), (2,3) at the mean of their ends,
 * so the geometry is the vertices' affine map; thermal form, FP64, exact
 * integration, up to 128 neighbours per node), 8 (Q2S_QUAD: the 8-node
 * serendipity quadrilateral of the paper's 2D thermal case; vertices
 * a = i + 2j at reference corner (2i-1, 2j-1), then the midpoints of the x
 * edges (at y = 2j-1) 4 + j and of the y edges (at x = 2i-1) 6 + i, at the
 * mean of their ends, so the geometry is the vertices' bilinear map;
 * thermal form, FP64, 3 x 3 Gauss).  Triangles are
 * counter-clockwise.  For the flow form, pconn [n_elems][3] gives the P1
 * pressure nodes (the element's vertices in a 0..n_pnodes-1 numbering). */
typedef struct {
    int32_t dim;
    int32_t elem;            /* mf_elem */
    int64_t n_nodes;
    int64_t n_elems;
    const double *coords;
    const int32_t *conn;
    int64_t n_pnodes;        /* flow only, else 0 */
    const int32_t *pconn;    /* flow only, else NULL */
} mf_mesh_desc;

/* Coefficients of a form (Sec. 4.1-4.3).  elem_coef [n_elems]: the
 * conductivity k (thermal) or Young's modulus E (elasticity); ignored by the
 * flow form.  source: thermal f = source[0]; elasticity body force b[3].
 * advect [2][n_nodes]: nodal advecting velocity of the flow form; for the
 * Navier-Stokes form (MF_FORM_NS) the current state [u1 | u2 | p]
 * (2 n_nodes + n_pnodes), with the stabilisation parameters tau_m, tau_c of
 * the SUPG terms (constants, Sec. 4.3).  bc_mask
 * [n_dofs] (u8, nonzero = Dirichlet) and bc_val [n_dofs] f64 may be NULL
 * (no constraint).  Dirichlet dofs are eliminated symmetrically: row and
 * column zeroed in the pattern, K[g][g] = 1, d[g] = bc_val[g], and
 * d[i] -= K[i][g] bc_val[g] on the other rows. */
typedef struct {
    const double *elem_coef;
    double nu;               /* Poisson ratio (elasticity) */
    double visc;             /* dynamic viscosity mu (flow) */
    double rho;              /* density (flow) */
    double source[3];
    const double *advect;
    const uint8_t *bc_mask;
    const double *bc_val;
    double tau_m, tau_c;     /* SUPG parameters (MF_FORM_NS) */
} mf_coeffs;

/* CSR view.  row_ptr [n_rows+1] int64, col_idx [nnz] int32 ascending within a
 * row, the diagonal always present.  Owned by the pattern; values [nnz] is a
 * caller buffer. */
typedef struct {
    int64_t n_rows;
    int64_t nnz;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    double *values;
} mf_csr;

typedef struct {
    int32_t solver;          /* mf_solver */
    int32_t restart;         /* GMRES restart length m (e.g. 50) */
    double tol;              /* stop at ||d - K x||_2 <= tol ||d||_2 */
    int64_t max_iter;
    const double *precond_diag; /* GMRES: device [n] diagonal P (x = P^-1 y);
                                   NULL = diag(K).  PCG always uses diag(K). */
    int32_t check_every;     /* host reads the residual every k iterations (>= 1) */
    double inner_tol;        /* MF_SOLVER_PCG_REFINED: relative residual of each FP32
                                inner solve (0: 1e-4) */
    const mf_flow_mg *flow_mg; /* MF_SOLVER_GMRES_FLOW_MG: the preconditioner hierarchy */
} mf_solver_opts;

typedef struct {
    int64_t iterations;      /* PCG / GMRES iterations; refined PCG: inner FP32 iterations */
    double rel_residual;     /* true ||d - K x|| / ||d|| recomputed at exit (FP64) */
    int32_t converged;
    int64_t refinements;     /* MF_SOLVER_PCG_REFINED: FP64 correction steps */
} mf_solve_info;

/* Validates and wraps a mesh (Block B-1).  Checks on the device that every
 * connectivity entry is in range and detJ > 0 at every quadrature point;
 * synchronises the stream.  Keeps the caller's device pointers (they must
 * outlive the handle); coordinates and connectivity must not change while
 * patterns or facet sets of the mesh live (those keep data derived from
 * them).  Errors: MF_ERR_INVALID_ARG, MF_ERR_BAD_MESH,
 * MF_ERR_NONFINITE, MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_mesh_create(const mf_mesh_desc *desc, void *stream, mf_mesh **out);
mf_status mf_mesh_destroy(mf_mesh *mesh);

/* Builds the sparsity pattern of a form on a mesh (Block A-3 symbol pairs x
 * Block B-1 unique control-point pairs -> Block B-4 sparse ids), as CSR with
 * ascending columns plus the element -> entry maps the assembly uses.  The
 * flow form has the blocks u1-u1, u2-u2, u-p, p-u and the p-p diagonal; no
 * u1-u2 block.  The Navier-Stokes form (MF_FORM_NS) has every block: u1-u2
 * (the convective derivative) and the full P1 x P1 p-p block (the SUPG
 * pressure term).  Elasticity takes Q1 and Q2S bricks (dof 3 n + c, 3 x 3
 * blocks per node pair).  Synchronises the stream.  Errors:
 * MF_ERR_INVALID_ARG, MF_ERR_UNSUPPORTED (a form the element does not
 * carry; more than 64 neighbours (128 for Q2S) or 32 incident elements per
 * node), MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_pattern_build(const mf_mesh *mesh, int32_t form, void *stream, mf_pattern **out);
/* Fills n_rows, nnz, row_ptr, col_idx (device pointers owned by the pattern);
 * values = NULL. */
mf_status mf_pattern_csr(const mf_pattern *pattern, mf_csr *out);
/* Copies the pattern's CSR arrays into caller device buffers row_ptr
 * [n_rows+1] (int64) and col_idx [nnz] (int32), asynchronously on the stream. */
mf_status mf_pattern_copy_csr(const mf_pattern *pattern, int64_t *row_ptr, int32_t *col_idx, void *stream);
mf_status mf_pattern_destroy(mf_pattern *pattern);

/* Assembles K and d (Block D-2 residual and D-3 tangent, sparse value and
 * residual arrays cleared first) for one form: per element quadrature of the
 * form (Sec. 2.1), then a deterministic sum into CSR (no float atomics: two
 * calls give bit-identical K and d), then the Dirichlet elimination.
 * K->values [nnz] and d [n_rows] are caller device buffers.  prec =
 * MF_PREC_FP64: FP64 element blocks summed node by node in ascending element
 * order.  prec = MF_PREC_MIXED (elasticity on Q1 only, any nu in (-1, 0.5)):
 * tensor-core element contraction on BF16 slices of the mu-scaled gradients,
 * blocks added as exact 64-bit fixed-point integers (integer atomics, so the
 * order does not change the bits) at a scale taken from the current
 * coordinates and coefficients in every call, then K = r A + A^T + I tr A
 * per CSR block with r = lambda/mu = 2nu/(1-2nu) as an exact 53-bit
 * multiplier, converted once to FP64; K within about 2^-40 of the row scale
 * of the FP64 result.  Errors:
 * MF_ERR_INVALID_ARG, MF_ERR_UNSUPPORTED, MF_ERR_CUDA; non-finite
 * coefficients (on the mixed path also a non-finite coordinate, found by
 * the pass that sets the fixed-point scale) are latched (MF_ERR_NONFINITE). */
mf_status mf_assemble(int32_t form, const mf_mesh *mesh, const mf_pattern *pattern,
                      const mf_coeffs *coeffs, int32_t prec, mf_csr *K, double *d, void *stream);
/* form = MF_FORM_NS (prec FP64, on a pattern built for MF_FORM_NS: every
 * block, u1-u2 and the full p-p block included) linearises the steady
 * Navier-Stokes form with SUPG at the state x = coeffs->advect (Sec. 4.3
 * domain form, Newton of Sec. 2.1):
 *   r_(a,i) = int -rho (grad N_a . u) u_i - d_i N_a p + mu grad N_a . grad u_i
 *             + tau_m rho (grad N_a . u) Rm_i + tau_c d_i N_a Rc,
 *   r_b     = int M_b Rc + tau_m grad M_b . Rm,
 *   Rm = rho (u . grad) u + grad p - mu lap u,  Rc = div u,
 * K = dr/dx (the tangent, by hand-derived derivatives) and d = -r, so that
 * K dx = d is the Newton step.  Dirichlet dofs g get the increment data
 * bc_val[g] - x[g] with the same symmetric elimination as the other forms.
 * Integrals by a collapsed 4 x 4 Gauss rule, exact for every integrand on
 * straight-sided triangles. */
/* form = MF_FORM_CAPACITY (prec FP64, on a thermal pattern) assembles the
 * capacity matrix of the rate term -C(T, T_t) of Sec. 4.1, K[a][b] =
 * sum_e C_e int_e N_a N_b with C_e = elem_coef[e], exactly on affine elements
 * (P1, P2, P2T: closed forms; Q1: 2 x 2 x 2 Gauss; Q2S_QUAD: 3 x 3 Gauss;
 * not provided on Q2S bricks), and d = 0 (then the Dirichlet elimination if
 * bc_mask is given). */

/* ---- Boundary (facet) terms -----------------------------------------------
 * A boundary condition is the domain physics one dimension lower (Sec. 2.2):
 * the convection term h(T, T_env - T) of Sec. 4.1 and the loaded boundary
 * (d_i, sigma^l_ij n_j) of Sec. 4.2, integrated over facets.  A facet is a
 * local face of a mesh element:
 *  - triangle face f is the edge from vertex f to vertex (f + 1) % 3; on P2
 *    the midpoint node 3 + f is its third node.  Edges are straight.
 *  - hexahedron face 2d + s is the face where reference coordinate d equals
 *    2s - 1; its nodes are the element nodes a with bit d of a equal to s,
 *    ascending, and its map is bilinear in the other two reference
 *    coordinates.  n is the outward unit normal.
 *  - quadrilateral (Q2S_QUAD) face f is an edge, counter-clockwise: nodes
 *    (0, 1, 4), (1, 3, 7), (3, 2, 5), (2, 0, 6) for f = 0..3 (the two ends,
 *    then the midpoint), integrated as a straight P2 edge.
 *  - tetrahedron (P2T) face i is the face opposite vertex i; its nodes are
 *    the three vertices in outward order (1,2,3), (0,3,2), (0,1,3), (0,2,1)
 *    for i = 0..3, then the midpoints of its edges (0,1), (1,2), (2,0) in
 *    face order; the face is flat.  Thermal (convection) only.
 *  - 20-node brick (Q2S) face 2d + s: its 4 vertices as on the Q1 brick (face
 *    node i + 2j, i and j the bits of the face axes d1 < d2), then the edge
 *    midpoints in the 8-node quadrilateral's order: the d1 edges at bit
 *    d2 = j (4 + j), the d2 edges at bit d1 = i (6 + i); the 8-node
 *    serendipity basis on the vertices' bilinear map (straight edges).
 *    Convection and the loaded boundary (the cantilever loads of Sec. 4.2).
 * Quadrature: Gauss-Legendre with 2 (P1) or 3 (P2) points per edge, exact for
 * the edge mass matrix; 2 x 2 Gauss on a Q1 face, 3 x 3 on an 8-node face; on
 * a tetrahedron face the exact P2 triangle mass matrix and load.  Radiation
 * (mf_genalpha_run) is not provided on tetrahedron and 8-node brick faces
 * (MF_ERR_UNSUPPORTED). */
typedef struct mf_facets mf_facets;

/* Wraps n_facets facets (elem [n_facets] int32 parent elements, face
 * [n_facets] u8 local faces; device arrays read during this call only) of a
 * mesh for a thermal or elasticity pattern.  Builds on the device the facets
 * incident to every boundary node in ascending facet order and, for the
 * thermal form, each facet node's position in the node's CSR row, and
 * keeps each facet's geometry (the coefficient-free factors of the terms
 * below).  n_facets = 0 is valid (no boundary terms).  Synchronises the stream.
 * Errors: MF_ERR_INVALID_ARG (NULL, negative count, flow pattern, pattern of
 * another mesh), MF_ERR_BAD_MESH (element or face out of range),
 * MF_ERR_UNSUPPORTED (more than 32 facets at one node), MF_ERR_OOM,
 * MF_ERR_CUDA. */
mf_status mf_facets_create(const mf_mesh *mesh, const mf_pattern *pattern, int64_t n_facets,
                           const int32_t *elem, const uint8_t *face, void *stream, mf_facets **out);
mf_status mf_facets_destroy(mf_facets *facets);

/* Coefficients of the boundary terms, per facet (device arrays).  Thermal:
 * h [n_facets] convective coefficient, t_env [n_facets] ambient temperature.
 * Elasticity: stress [n_facets][3][3] row-major sigma^l, the facet's load
 * being sigma^l n.  bc_mask / bc_val: the Dirichlet data the system was
 * assembled with (both NULL: none). */
typedef struct {
    const double *h;
    const double *t_env;
    const double *stress;
    const uint8_t *bc_mask;
    const double *bc_val;
} mf_facet_coeffs;

/* Adds the boundary terms of the facets to a system assembled by
 * mf_assemble on the same pattern (values [nnz], d [n_rows], in place):
 *   thermal     K[a][b] += sum_q w_q |J_q| h N_a N_b,
 *               d[a]    += sum_q w_q |J_q| h T_env N_a;
 *   elasticity  d[3a+i] += sum_q w_q N_a sigma_ij (n |J|)_j
 * over the facets of node a, |J| the facet's length or area element.  Rows
 * of Dirichlet dofs stay as assembled; a term in the column of a Dirichlet
 * dof g goes to the right-hand side, d[a] -= term * bc_val[g].  The result is
 * that of assembling domain and boundary terms together before the
 * elimination, up to the rounding order.  Each node sums its facets in
 * ascending facet order: two calls give identical bits.  Errors:
 * MF_ERR_INVALID_ARG, MF_ERR_CUDA; non-finite coefficients are latched
 * (MF_ERR_NONFINITE). */
mf_status mf_assemble_boundary(const mf_facets *facets, const mf_facet_coeffs *coeffs, mf_csr *K, double *d,
                               void *stream);

/* ---- Generalised-alpha time stepping ---------------------------------------
 * Sec. 2.1 (Eq. time_constraints, time_effective) and Blocks C, D of Sec. 2.2
 * for the linear conduction system with capacity: per dof the value phi, its
 * rate u and second rate a; increments dphi, du, da tied by the constraints
 * dphi = dt (u + b1 du), du = dt (a + b2 da); residual at the effective
 * values phi~ = phi + c1 dphi, u~ = u + c2 du (a~ = a + c3 da does not enter
 * a first-order form):  d = F - K phi~ - M u~;  tangent (Block D-3) T = c1 K +
 * c2 / (b1 dt) M. */
typedef struct {
    double b1, b2, c1, c2, c3;
} mf_genalpha_params;

/* Parameters of the first-order generalised-alpha method of Jansen, Whiting
 * and Hulbert (2000) with high-frequency spectral radius rho_inf in [0, 1]:
 * alpha_m = (3 - rho_inf) / (2 (1 + rho_inf)), alpha_f = 1 / (1 + rho_inf),
 * gamma = 1/2 + alpha_m - alpha_f; b1 = b2 = gamma, c1 = alpha_f,
 * c2 = c3 = alpha_m.  Second-order accurate, unconditionally stable.
 * Errors: MF_ERR_INVALID_ARG. */
mf_status mf_genalpha_params_from_rho(double rho_inf, mf_genalpha_params *out);

/* Runs `steps` time steps of length dt.  K: CSR of the stiffness (values
 * with any convection terms, no Dirichlet elimination); M_values [nnz]: the
 * capacity matrix on the same pattern; F [n]: the load; bc_mask / bc_val
 * [n] (or NULL): Dirichlet dofs, which keep phi = bc_val and u = a = 0.
 * phi, u, a [n] (device): the state at t on entry (u should be the
 * consistent rate, M u = F - K phi on free rows) and at t + steps dt on exit.
 * Each step: C-1 apply the last increments, C-2 da = 0, C-3 du = dt a,
 * dphi = dt (u + b1 du); then Newton sub-steps (Block D): residual d at the
 * effective values, stop when ||d||_2 <= newton_tol ||d_0||_2 (d_0: the
 * step's first residual) or ||d|| <= 1e-13 (||F|| + ||K phi~|| + ||M u~||)
 * on the free rows; else solve T x = d by Jacobi-PCG to pcg_tol (relative),
 * dphi += x, du = (dphi / dt - u) / b1, da = (du / dt - a) / b2.  The norms
 * are fixed-order sums: runs are bit-reproducible.  newton_its, pcg_its
 * (host [steps], may be NULL): solves and PCG iterations per step.
 * Radiation (Sec. 4.1, e_m sigma^b (T, T_env^4 - T^4)): rad (may be NULL) is
 * a facet set of K's thermal pattern with rad_es [n_facets] = e_m sigma^b
 * and rad_tenv [n_facets]; the residual then uses F + R(phi~), R_a =
 * sum_f es int N_a (T_env^4 - T~^4) (facet rule), also inside the rounding
 * floor, and the tangent gains c1 K_rad, K_rad[a][b] = sum_f 4 es int N_a
 * N_b T~^3: full Newton.
 * Synchronises the stream every sub-step.  Errors: MF_ERR_INVALID_ARG,
 * MF_ERR_NOT_CONVERGED (a step used max_newton solves, or a PCG solve hit
 * pcg_max_iter), MF_ERR_NONFINITE, MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_genalpha_run(const mf_csr *K, const double *M_values, const double *F, const uint8_t *bc_mask,
                          const double *bc_val, const mf_facets *rad, const double *rad_es, const double *rad_tenv,
                          double *phi, double *u, double *a, const mf_genalpha_params *prm, double dt,
                          int64_t steps, double newton_tol, int32_t max_newton, double pcg_tol, int64_t pcg_max_iter,
                          int64_t *newton_its, int64_t *pcg_its, void *stream);

/* Consistent initial rate: solves M u = F + R(phi) - K phi on the free rows
 * (u = 0 on Dirichlet rows; R the radiation loads, if rad is given) by
 * Jacobi-PCG to pcg_tol.  Arguments as mf_genalpha_run; u [n] device
 * output.  Synchronises the stream.  Errors: MF_ERR_INVALID_ARG,
 * MF_ERR_NOT_CONVERGED, MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_genalpha_initial_rate(const mf_csr *K, const double *M_values, const double *F, const uint8_t *bc_mask,
                                   const mf_facets *rad, const double *rad_es, const double *rad_tenv,
                                   const double *phi, double *u, double pcg_tol, int64_t pcg_max_iter, void *stream);

/* Pressure-mass diagonal of the flow form, out[a] = sum_e sum_q w detJ M_a^2
 * over P1 pressure node a (for the block-diagonal GMRES preconditioner).
 * out [n_pnodes] device.  Errors: MF_ERR_INVALID_ARG, MF_ERR_CUDA. */
mf_status mf_pressure_mass_diag(const mf_mesh *mesh, const mf_pattern *pattern, double *out,
                                void *stream);

/* Block-diagonal preconditioner of the flow system for GMRES:
 * out[r] = K[r][r] on velocity rows, p_scale * Mp[n] on the pressure row of
 * P1 node n (Mp the pressure-mass diagonal), 1 on constrained dofs.
 * out [n_rows] device.  Errors: MF_ERR_INVALID_ARG, MF_ERR_CUDA. */
mf_status mf_flow_precond(const mf_mesh *mesh, const mf_pattern *pattern, const mf_csr *K,
                          const uint8_t *bc_mask, double p_scale, double *out, void *stream);

/* Preconditioner of the flow system (Sec. 4.3 Picard form on the Taylor-Hood
 * P2-P1 split-square grids, dofs [u1 | u2 | p]) for MF_SOLVER_GMRES_FLOW_MG:
 * the block upper-triangular M = [A B^T; 0 S] applied exactly in its block
 * structure, S = diag(M_p) / visc (pressure mass over the viscosity, 1 on a
 * constrained pressure dof), and A^-1 replaced by one geometric multigrid
 * V-cycle (2 + 2 damped Jacobi sweeps with weight 4 / (3 lambda_max(D^-1 A)),
 * 60 on the coarsest grid, P2 interpolation between grids and its transpose,
 * constrained velocity dofs held).  K[l], bc_mask[l] (device, [n_rows of
 * level l]) are the flow systems assembled by mf_assemble on the grids of
 * cells[l] cells per side, finest first, each grid halving the previous one
 * (levels <= 12); pmass (device [n_pnodes]) is mf_pressure_mass_diag of the
 * finest grid.  The hierarchy copies what it needs (the velocity blocks,
 * masks); the caller keeps K[0] for the solve.  Synchronises the stream.
 * Errors: MF_ERR_INVALID_ARG (levels, sizes), MF_ERR_NONFINITE (a zero
 * diagonal), MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_flow_mg_create(int32_t levels, const mf_csr *const *K, const int64_t *cells,
                            const uint8_t *const *bc_mask, const double *pmass, double visc, void *stream,
                            mf_flow_mg **out);
mf_status mf_flow_mg_destroy(mf_flow_mg *mg);

/* Solves K x = d (Block D-4; the paper leaves the solver open): Jacobi-PCG
 * (symmetric positive K), right-preconditioned restarted GMRES(m) with
 * classical Gram-Schmidt applied twice, or (MF_SOLVER_PCG_REFINED) FP64
 * iterative refinement around an FP32 Jacobi-PCG: the residual r = d - K x
 * is formed in FP64 with K as given, each correction K z = r / ||r|| is
 * solved on an FP32 copy of K with FP32 vectors to inner_tol, and x += ||r|| z
 * in FP64, until ||d - K x|| <= tol ||d|| (max_iter caps the inner
 * iterations; the refinement needs kappa(K) 2^-24 well below 1; three
 * refinements in a row that do not halve the residual end the solve with
 * MF_ERR_NOT_CONVERGED: the FP64 residual has reached its rounding floor
 * above tol), or
 * (MF_SOLVER_GMRES_FLOW_MG) right-preconditioned GMRES(restart) with the
 * flow hierarchy opts->flow_mg (mf_flow_mg_create).  x holds x0 on entry (a warm start
 * resumes a previous solve) and the solution on exit.  Synchronises the
 * stream.  Returns MF_ERR_NOT_CONVERGED (x = last iterate, info filled) at
 * max_iter, MF_ERR_NONFINITE for a non-finite d or a breakdown, and any
 * latched device error.  info may be NULL. */
mf_status mf_solve(const mf_csr *K, const double *d, double *x, const mf_solver_opts *opts,
                   mf_solve_info *info, void *stream);

/* Newton-Raphson (Sec. 2.1) on the Navier-Stokes form with SUPG: x (device
 * [2 n_nodes + n_pnodes], the state; entries of Dirichlet dofs are set to
 * bc_val first) is updated by steps K dx = -r (mf_assemble with MF_FORM_NS,
 * then mf_solve with *lin: GMRES, or GMRES with a flow hierarchy of
 * mf_flow_mg_create, e.g. built from the Stokes systems of the grids, whose
 * block-triangular preconditioner takes the tangent's own velocity-pressure
 * coupling) until the residual on the free dofs
 * satisfies ||r_free|| <= newton_tol max(1, ||r_free(x0)||), at most
 * max_newton steps.  coeffs->advect is ignored (x is the state).  resid_hist
 * (host, max_newton + 1 entries, may be NULL) receives ||r_free|| before each
 * step; *n_steps the number of steps taken.  Synchronises the stream.
 * Returns MF_ERR_NOT_CONVERGED at max_newton or when a linear solve fails to
 * converge, and the errors of mf_assemble and mf_solve. */
mf_status mf_ns_newton(const mf_mesh *mesh, const mf_pattern *pattern, const mf_coeffs *coeffs, double *x,
                       double newton_tol, int32_t max_newton, const mf_solver_opts *lin, double *resid_hist,
                       int32_t *n_steps, void *stream);

/* Jacobi-PCG like mf_solve (same kernels and stopping rule), but it makes no
 * device allocation: no cudaMalloc, no cudaFree, no graph, stream or event
 * creation.  It is meant for callers that cannot allocate during a solve, e.g.
 * a framework that reserved all device memory for its own pool at start-up,
 * or a latency-critical loop where an allocation would synchronise the device.
 * The paper has no counterpart; this entry exists for those callers.
 * Work memory is one file-scope __device__ array holding four vectors of
 * MF_NOALLOC_MAX_ROWS doubles (about 32 MB), kept by every GPU that loads the
 * library until the process exits.  Systems with more rows are rejected with
 * MF_ERR_INVALID_ARG.  The first call on a device looks up the array's device
 * address (set-up, once per device, with that device current); make that
 * first call before any stream capture.  Every call shares the array and
 * keeps the last call's contents (the state is reset at entry), so calls that
 * overlap on the GPU (several streams or host threads) race: serialise them.
 * x holds x0 on entry and the solution on exit; info may be NULL.
 * Synchronises the stream.  Errors: as mf_solve. */
#define MF_NOALLOC_MAX_ROWS (1 << 20)
mf_status mf_solve_pcg_noalloc(const mf_csr *K, const double *d, double *x, double tol, int64_t max_iter,
                               int32_t check_every, mf_solve_info *info, void *stream);

/* y = K x (device pointers). */
mf_status mf_spmv(const mf_csr *K, const double *x, double *y, void *stream);

/* Per-kernel timing with CUDA events (tracing).  While enabled, every kernel
 * launched by mf_assemble is bracketed by two events recorded on the call's
 * stream.  mf_kernel_times() synchronises those events, writes
 * "name count total_ms\n" lines (one per kernel name) into buf (NUL
 * terminated, truncated to len) and clears the counters.  Host-side only; no
 * effect on results.  Errors: MF_ERR_INVALID_ARG, MF_ERR_CUDA. */
mf_status mf_set_kernel_timing(int32_t enable);
mf_status mf_kernel_times(char *buf, size_t len);

/* ---- Batched assembly (many thermal problems in one launch) -------------
 * Many independent thermal problems (Sec. 4.1 form) of uneven size and mixed
 * element order (P1, P2, Q1), each with its own mesh, pattern, coefficients
 * and output buffers, are assembled by one persistent launch over a queue of
 * (problem, tile) work items: element tiles sorted by element type, and node
 * tiles of the fixed-order gather, each problem's node tiles queued after its
 * element tiles (they wait, bounded, for them: MF_ERR_TIMEOUT in the status
 * word if the wait gives up).  A counter reset and the launch are captured in
 * a CUDA graph at the first mf_batch_assemble and replayed.  Each problem's K
 * and d are bitwise equal to mf_assemble's.  Tiling: elements per tile,
 * threads per block, nodes per gather tile, blocks per SM (grid size). */
typedef struct mf_batch mf_batch;
typedef struct {
    int32_t elem_tile;
    int32_t elem_block;      /* multiple of 32, <= 256 */
    int32_t node_tile;
    int32_t grid_per_sm;
} mf_batch_tiling;
/* meshes/patterns [n] (thermal patterns of those meshes), coeffs [n] (host
 * array of device-pointer structs), values[i] [nnz_i] and d[i] [n_rows_i]
 * device buffers; all must outlive the batch.  Errors: MF_ERR_INVALID_ARG,
 * MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_batch_create(int32_t n, const mf_mesh *const *meshes, const mf_pattern *const *patterns,
                          const mf_coeffs *coeffs, double *const *values, double *const *d, mf_batch **out);
mf_status mf_batch_set_tiling(mf_batch *batch, const mf_batch_tiling *tiling);
mf_status mf_batch_get_tiling(const mf_batch *batch, mf_batch_tiling *tiling);
/* Autotuner: times candidate tilings (3 graph replays each) on this batch and
 * keeps the fastest; with cache_path (a small JSON file, may be NULL) a tiling
 * found earlier for the same batch signature is reused without timing, and a
 * new result is stored.  Synchronises the stream. */
mf_status mf_batch_autotune(mf_batch *batch, const char *cache_path, void *stream, mf_batch_tiling *chosen);
/* Assembles every problem of the batch (one graph launch, asynchronous). */
mf_status mf_batch_assemble(mf_batch *batch, void *stream);
mf_status mf_batch_destroy(mf_batch *batch);

/* ---- Learned preconditioner correction (3D CNN) -------------------------
 * Not in the paper: a growth line of the hot path.  A 4-layer 3x3x3
 * convolution network (2 -> 16 -> 16 -> 16 -> 1 channels, ReLU after the first
 * three, zero padding) on the node grid (nz, ny, nx) of a structured Q1 thermal
 * problem (node v = (z ny + y) nx + x).  BF16 weights and activations, FP32
 * accumulation, FP32 master weights and AdamW moments for training.  Inputs
 * per node: (r / max|r|, log k_nodal / 2) in BF16.  Used as
 *   z = D^-1 r + max|r| (1 - mask) CNN(r / max|r|, log k)
 * inside flexible CG, falling back to z = D^-1 r when z . r <= 0.
 * Parameters: mf_cnn_num_params() floats, layer by layer [w (co, ci, 27) | b (co)],
 * offset index o = (dz+1) 9 + (dy+1) 3 + (dx+1). */
typedef struct mf_cnn mf_cnn;
int64_t mf_cnn_num_params(void);
/* init: host array of mf_cnn_num_params() floats (initial weights). */
mf_status mf_cnn_create(const float *init, mf_cnn **out);
mf_status mf_cnn_destroy(mf_cnn *cnn);
mf_status mf_cnn_get_params(const mf_cnn *cnn, float *host, int64_t n);
mf_status mf_cnn_get_grads(const mf_cnn *cnn, float *host, int64_t n);
/* x: device BF16 [B][nv][2], 4-byte aligned (a node's two channels are read
 * as one word); y: device FP32 [B][nv].  MF_ERR_INVALID_ARG for a misaligned
 * x or B nv > (2^31 - 1) / 16 (the same bound for training and FCG). */
mf_status mf_cnn_forward(mf_cnn *cnn, int32_t B, int32_t nz, int32_t ny, int32_t nx, const void *x, float *y,
                         void *stream);
/* Gradients of sum(gy * CNN(x)) into the gradient buffer (read with
 * mf_cnn_get_grads); runs the forward pass first.  All four layers' weight
 * gradients and the 16-channel input gradients are tensor-core GEMMs over the
 * nodes (BF16 operands, FP32 accumulation); the gradients passed between
 * layers are masked by the ReLU and rounded to BF16.  x as mf_cnn_forward. */
mf_status mf_cnn_backward(mf_cnn *cnn, int32_t B, int32_t nz, int32_t ny, int32_t nx, const void *x,
                          const float *gy, void *stream);
/* One AdamW step (lr > 0; lr = 0 only computes the loss and gradients) on B
 * samples of systems sharing the pattern of K: kvals[b] the values of system
 * b, r[b] its residual, x[b] its network input (device pointers); the Jacobi
 * part uses diag(K_b).  loss (host): without err, mean_b ||K_b z_b - r_b||^2 /
 * ||r_b||^2; with err[b] = K_b^-1 r_b (the error of the iterate), the energy
 * left after one optimally scaled step along z_b,
 * mean_b 1 - (z_b . K_b err_b)^2 / ((z_b . K_b z_b)(err_b . K_b err_b)). */
mf_status mf_cnn_train_step(mf_cnn *cnn, int32_t B, int32_t nz, int32_t ny, int32_t nx, const mf_csr *K,
                            const double *const *kvals, const double *const *r, const double *const *err,
                            const void *const *x, const uint8_t *mask, float lr, float weight_decay, double *loss,
                            void *stream);
/* Nodal mean of log k over the cells of the (nz-1)(ny-1)(nx-1) cell grid. */
mf_status mf_cnn_node_logk(int32_t nz, int32_t ny, int32_t nx, const double *kcell, float *out, void *stream);
/* Network input from a residual: x [n][2] BF16 = (r / max|r|, logk / 2). */
mf_status mf_cnn_input(int64_t n, const double *r, const float *logk, void *x_bf16, void *stream);
/* y = a x + b y on device vectors of length n. */
mf_status mf_axpby(int64_t n, double a, const double *x, double b, double *y, void *stream);
/* Flexible CG (Notay 2000) preconditioned by the CNN correction with the
 * Jacobi fallback, each new direction K-orthogonalised against the last
 * m_dirs directions (1 <= m_dirs <= 256; 1 is the classic flexible CG); x holds x0 on
 * entry.  fallbacks (may be NULL) counts the iterations that fell back to
 * Jacobi.  Work space: (2 m_dirs + 4) vectors of n doubles.  Errors: as
 * mf_solve, MF_ERR_INVALID_ARG for m_dirs outside [1, 256]. */
mf_status mf_solve_fcg_cnn(const mf_csr *K, const double *d, double *x, mf_cnn *cnn, int32_t nz, int32_t ny,
                           int32_t nx, const float *logk, const uint8_t *mask, double tol, int64_t max_iter,
                           int32_t m_dirs, mf_solve_info *info, int64_t *fallbacks, void *stream);

/* Synchronises the stream, returns and clears the latched device status. */
mf_status mf_sync_status(void *stream);

/* Thread-local message of the last failing call ("" if none). */
const char *mf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MF_H */
