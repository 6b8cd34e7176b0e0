/*
 * mmncg -- preconditioned nonlinear conjugate gradient (NCG) minimisation of
 * the micromagnetic energy on P1 tetrahedral meshes, on one GB300 GPU.
 *
 * The method is that of Exl, Fischbacher, Kovacs, Oezelt, Gusenbauer and
 * Schrefl, "Preconditioned nonlinear conjugate gradient method for
 * micromagnetic energy minimization" (arXiv:1801.03690):
 *   - Eq. (energy), Sec. 2.2: F(m) = 1/2 m^T C m - 1/2 h_d^T M m - h_ext^T M m,
 *     C = C_A + C_K (exchange + anisotropy), magnetostatics from a scalar
 *     potential in an air box (Sec. 3.1);
 *   - Algorithm 4 with beta*ZA (Sec. 2.2), minimising F(N m) with the
 *     projected gradient of Eqs. (nablaLF), (proj), (opt2);
 *   - the sparse approximate-Hessian preconditioner, Eq. (precond), solved by
 *     Algorithm 1 with Jacobi diag(C_A) and the exits li1-li3 (Sec. 3.1);
 *   - the stopping rules t1-t3 (Sec. 3.1).
 *
 * Conventions (all entry points):
 *   - Every call returns an int status: MM_OK (0), a negative MM_ERR_* code,
 *     or a positive soft status (MM_NOT_CONVERGED, MM_STALLED).
 *     mm_last_error() gives a message for the last failing call.
 *   - Inputs are SI: coordinates in metres, Ms in A/m, A in J/m, K1 in J/m^3,
 *     applied fields as mu0*H in tesla.  Energies are returned in joules.
 *     Internally (and for the stopping rules t1-t3, which compare energies
 *     against 1) lengths are in nm and energies in units of
 *     mu0*Mref^2*(1 nm)^3, Mref = the largest Ms in the material table.
 *   - Host arrays passed in are copied; the caller keeps ownership.  Host
 *     output arrays are written in full before the call returns.
 *   - Calls with the suffix _dev take device pointers owned by the caller
 *     (never freed by the library) and enqueue work on the context's stream
 *     without synchronising, unless stated otherwise.
 *   - Per-node arrays are indexed by the caller's node ids, row-major [n][3].
 *     Only magnetic nodes (vertices of a tetrahedron with Ms > 0) carry m;
 *     other rows are ignored on input and written as 0 on output.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef MMNCG_H
#define MMNCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MM_OK = 0,
    MM_NOT_CONVERGED = 1,        /* max_iter reached before t1-t3 held         */
    MM_STALLED = 2,              /* line search found no decrease; m unchanged */
    MM_ERR_ARG = -1,             /* invalid argument (NULL, size, parameter)   */
    MM_ERR_MESH = -2,            /* invalid mesh: index, degenerate tet, ...   */
    MM_ERR_OOM = -3,             /* device allocation failed                   */
    MM_ERR_CUDA = -4,            /* CUDA runtime error                         */
    MM_ERR_NONFINITE = -5,       /* NaN/Inf met in an energy or reduction      */
    MM_ERR_DEVICE_TIMEOUT = -6,  /* a device-side barrier wait ran out         */
    MM_ERR_STATE = -7            /* call out of order (e.g. no mesh uploaded)  */
};

typedef struct mm_ctx mm_ctx;

/* One row of the material table (one per region label).  Ms = 0 marks a
 * non-magnetic region (air).  The easy axis need not be normalised. */
typedef struct {
    double Ms;        /* saturation magnetisation, A/m                       */
    double A;         /* exchange constant, J/m                              */
    double K1;        /* uniaxial anisotropy constant, J/m^3                 */
    double axis[3];   /* easy axis                                           */
} mm_material;

typedef struct {
    int device;           /* CUDA device ordinal                                 */
    int blocks_per_sm;    /* solver kernel built for 2, 3 or 4 blocks/SM; 0 =    */
                          /* chosen at mm_upload_mesh: 4 above 2 M potential    */
                          /* unknowns, else 2                                   */
    void* stream;         /* cudaStream_t to run on; NULL = a private stream     */
} mm_options;

/* Parameters of Algorithm 4 (defaults from mm_default_params). */
typedef struct {
    double tau_F;          /* t1-t3 tolerance, Sec. 3.1 (default 1e-10)            */
    int jmax;              /* li1: max inner steps of the preconditioner (4)       */
    int max_iter;          /* NCG iteration cap per minimisation (10000)           */
    double theta_max;      /* line-search cap on max_i |alpha d_i| (0.1)           */
    double c1;             /* sufficient-decrease constant (1e-4)                  */
    int max_backtrack;     /* extra line-search evaluations allowed (10)           */
    int keep_last_term;    /* 1: keep the last term of Eq. (precond) (0)           */
    double poisson_tol;    /* relative residual of the potential solve (1e-10)     */
    int poisson_max_iter;  /* cap on potential-solve steps per evaluation (20000)  */
    int precision;         /* 0: FP64 throughout (0); 1: precision form -- the    */
                           /* potential solve runs Algorithm 1 in FP32 on the      */
                           /* correction equation K delta = r and refines the      */
                           /* residual r = D m - K phi in FP64 ("reliable          */
                           /* updates") until poisson_tol; the preconditioner     */
                           /* apply (Eq. precond) forms its H products and inner  */
                           /* CG vectors in FP32 (sums, step lengths and y FP64); */
                           /* energy, gradient, line search, beta and the         */
                           /* renormalisation stay FP64                            */
    double inner_tol;      /* FP32 residual drop that triggers an FP64 update (0.1)*/
    int max_refine;        /* cap on FP64 updates per potential solve (64)         */
    int amg;               /* precision form: 1 = precondition the FP32 solve with */
                           /* a smoothed-aggregation multigrid V-cycle (Sec. 3.1  */
                           /* uses algebraic multigrid there), 0 = Jacobi (0).    */
                           /* Needs the hierarchy mm_upload_mesh builds when      */
                           /* n_phi exceeds the dense coarse size; else Jacobi.   */
    int beta_rule;         /* direction update of Algorithm 3/4 (Sec. 2.1): 0 =   */
                           /* beta*ZA (default), 1 = beta*FR, 2 = beta*PRP        */
                           /* (Eqs. FRstar, PRPstar); the descent safeguard is     */
                           /* the same for all three                               */
    int poisson_sched;     /* 1: potential tolerance tied to t1 -- an iteration    */
                           /* whose previous energy decrease dF exceeds 100 times  */
                           /* the t1 threshold tau_F (1 + |F|) solves to           */
                           /* poisson_tol * sqrt(dF / threshold) / 10, at most     */
                           /* poisson_tol_max; otherwise (and on the first         */
                           /* iteration of a minimisation) to poisson_tol (0)      */
    double poisson_tol_max;/* loosest scheduled potential tolerance (1e-6)         */
} mm_params;

/* Counters of one call, in the columns of Table 1 plus the energy. */
typedef struct {
    int64_t evals;         /* function evaluations                                */
    int64_t nli;           /* nonlinear (NCG) iterations                          */
    int64_t li;            /* products with H inside the preconditioner solves    */
    int64_t mi;            /* products with K_phi inside the potential solves     */
    int64_t ls_extra;      /* evaluations spent backtracking in the line search   */
    int64_t mr;            /* FP64 refinement products (precision form; in mi)     */
    int32_t status;        /* MM_OK / MM_NOT_CONVERGED / MM_STALLED / error       */
    int32_t pad;
    double F;              /* energy at the returned state, J                     */
    double terms[4];       /* exchange, anisotropy, magnetostatic, Zeeman; J      */
    double F_internal;     /* energy in internal units (what t1-t3 see)           */
    double M[3];           /* sum_i w_i m_i / sum_i w_i (reduced magnetisation)   */
    /* branches taken (Sec. 3.1 li2, the descent safeguard of Alg. 4):        */
    int64_t li2;           /* preconditioner solves ended by negative curvature   */
    int64_t li2_first;     /* ... of them on the first inner step (y = g)         */
    int64_t restarts;      /* new directions whose y was replaced by g (g.d >= 0) */
    int64_t steepest;      /* directions that fell back to d = -g                 */
} mm_stats;

void mm_default_params(mm_params* p);

/* Create a context on a device.  opt may be NULL (device 0, private stream). */
int mm_create(mm_ctx** ctx, const mm_options* opt);
void mm_destroy(mm_ctx* ctx);
const char* mm_last_error(const mm_ctx* ctx);

/* Upload a tetrahedral mesh with per-tet region labels and a material table,
 * and assemble (on the GPU) every operator of Eq. (energy): the exchange
 * stiffness, the lumped anisotropy blocks and Ms weights, the scalar-
 * potential stiffness over magnet + air with phi = 0 on the outer surface of
 * the mesh, and the divergence coupling.  Sec. 2.2 and 3.1.  Couplings of
 * the potential stiffness that vanish in exact arithmetic but are assembled
 * as rounding residues (|a_ij| <= 1e-12 sqrt(a_ii a_jj); the face and body
 * diagonals of a rectilinear Kuhn lattice) are dropped: a product with the
 * stored operator differs from the assembled one by less than 1e-12
 * relative.
 *   xyz    [n_nodes][3] coordinates, m
 *   tets   [n_tets][4] node ids (either orientation; degenerate -> MM_ERR_MESH)
 *   region [n_tets] labels in [0, n_regions)
 * Resets m to +z on every magnetic node and the field to zero.  May be
 * called again to replace the mesh. */
int mm_upload_mesh(mm_ctx* ctx, int64_t n_nodes, const double* xyz,
                   int64_t n_tets, const int32_t* tets, const int32_t* region,
                   int32_t n_regions, const mm_material* materials);

/* Sizes: magnetic nodes, potential unknowns, nonzeros of the two graphs. */
int mm_sizes(const mm_ctx* ctx, int64_t* n_mag, int64_t* n_phi,
             int64_t* nnz_mag, int64_t* nnz_phi);

/* Multigrid hierarchy of the potential solve built by mm_upload_mesh
 * (Sec. 3.1 preconditions that solve with algebraic multigrid): *n_levels
 * smoothed levels L (0: none; mm_params.amg then runs Jacobi) and, for
 * l = 0..L, rows[l] the rows of level l (level L is the coarsest, solved
 * with a dense inverse), nnz_a[l] the nonzeros of its operator (level 0:
 * K_phi; level L: rows[L]^2 entries of the dense inverse) and, for l < L,
 * nnz_u[l] the nonzeros of U_l (the prolongation with the post-smoothing
 * step folded in, applied in the up phase) and nnz_p[l] those of the
 * smoothed prolongation P_l (its transpose restricts the pre-smoothed
 * residual in the down phase).  Any output may be NULL; at most
 * max_entries entries are written per array. */
int mm_amg_info(const mm_ctx* ctx, int32_t* n_levels, int64_t* rows, int64_t* nnz_a,
                int64_t* nnz_u, int64_t* nnz_p, int32_t max_entries);

/* Layout of the FP32 copy of K_phi the precision form streams (no
 * counterpart in the paper): *slices SELL-32 slices, *table_slices of them
 * with an offset table -- every row of such a slice couples to its own
 * index plus one of at most 8 offsets shared by the slice (the stencil of a
 * rectilinear lattice), so the slice stores values only -- and
 * *matrix_bytes, the bytes one FP32 product loads for the matrix (4 per
 * stored value in table slices, 8 per nonzero elsewhere, 32 per slice for
 * the table).  Any output may be NULL; MM_ERR_STATE without a mesh. */
int mm_k32_layout_info(const mm_ctx* ctx, int64_t* slices, int64_t* table_slices,
                       int64_t* matrix_bytes);

/* Host only (no GPU, no context): the FP32 layout that mm_upload_mesh
 * builds for K_phi (see mm_k32_layout_info), built for the symmetric matrix
 * A given in CSR (row_ptr [n+1], col [nnz], val [nnz], FP64; the caller
 * keeps ownership; A without its rounding residues, as upload stores it),
 * and applied in FP32 to x [n], writing y [n] = A x: every row summed over
 * its stored entries in the order the solver kernel sums them.  This is the
 * layout the kernel reads, exposed so that it can be checked without a GPU.
 * *table_slices and *matrix_bytes as in mm_k32_layout_info (may be NULL).
 * MM_ERR_ARG for null pointers, n < 1, decreasing row_ptr or a column
 * outside [0, n). */
int mm_k32_host_apply(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                      const float* x, float* y, int64_t* table_slices, int64_t* matrix_bytes);

/* Host only (no GPU, no context): build the multigrid hierarchy that
 * mm_upload_mesh builds for K_phi, for the symmetric positive definite
 * matrix A given in CSR (row_ptr [n+1], col [nnz], val [nnz], FP64; the
 * caller keeps ownership), and apply its V-cycle in FP64 to n_vec vectors
 * r [n_vec][n], writing z [n_vec][n].  This is the cycle the solver kernel
 * runs in FP32 (same set-up, same algebra), exposed so that the set-up can
 * be checked without a GPU.  Level 0 is aggregated on A's stored pattern
 * (values ignored) and computed with A without its rounding residues
 * (off-diagonal |a_ij| <= 1e-12 sqrt(a_ii a_jj)); every coarser level is the
 * Galerkin operator without its residues, columns ascending, aggregated on
 * its own pattern.  *n_levels and rows as in mm_amg_info; when
 * there is no hierarchy (n <= 1536, or the coarsening stalls) *n_levels = 0
 * and z is left untouched.  MM_ERR_ARG for null pointers, n < 1,
 * decreasing row_ptr or a column outside [0, n). */
int mm_amg_host_apply(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                      int32_t n_vec, const double* r, double* z, int32_t* n_levels,
                      int64_t* rows, int32_t max_rows);

/* Tile shape of the solver kernel's FP32 potential-solve products (no
 * counterpart in the paper; the results differ only by rounding):
 * rows_per_thread 1 or 2 (0 = default 2) -- SELL-32 rows each thread takes
 * at once in the level-0 products with K_phi and the smoothed prolongation,
 * two keeping twice the loads in flight; restrict_lanes 4, 8 or 16 (0 =
 * default 8) -- lanes that share one row of a restriction P^T (levels whose
 * rows average over 160 entries always take 32).  Kept by the context across
 * mm_upload_mesh; takes effect at the next solver launch.  MM_ERR_ARG for
 * other values. */
int mm_set_tiles(mm_ctx* ctx, int32_t rows_per_thread, int32_t restrict_lanes);

/* Magnetisation per node ([n_nodes][3]); normalised on entry (N m, Eq. opt2). */
int mm_set_magnetization(mm_ctx* ctx, const double* m);
int mm_get_magnetization(mm_ctx* ctx, double* m_out);
/* Device variants: m_dev [n_nodes][3] doubles on the context's device. */
int mm_set_magnetization_dev(mm_ctx* ctx, const double* m_dev);
int mm_get_magnetization_dev(mm_ctx* ctx, double* m_dev);

/* Uniform applied field mu0*H_ext in tesla (Eq. energy, last term). */
int mm_set_field(mm_ctx* ctx, const double mu0h[3]);

/* Minimise F at the current field from the current m by Algorithm 4 until
 * t1-t3 hold (Sec. 3.1).  The potential solve is warm-started from the last
 * potential.  p may be NULL (defaults).  Synchronises; fills *out (may be
 * NULL) and returns its status. */
int mm_minimize(mm_ctx* ctx, const mm_params* p, mm_stats* out);
/* Enqueue the same minimisation without waiting; read it with mm_get_stats. */
int mm_minimize_async(mm_ctx* ctx, const mm_params* p);
/* Wait for the context's stream and return the stats of the last
 * minimisation or evaluation. */
int mm_get_stats(mm_ctx* ctx, mm_stats* out);

/* Energy of m (host [n_nodes][3], or NULL for the current m) at the current
 * field: solves the potential (Sec. 3.1) and evaluates Eq. (energy).
 * F in J; terms (may be NULL) = exchange, anisotropy, magnetostatic, Zeeman. */
int mm_energy(mm_ctx* ctx, const double* m, const mm_params* p, double* F,
              double terms[4]);
/* Gradient of F at m (host or NULL = current), [n_nodes][3], internal units
 * (energy unit per unit of m).  projected = 1 returns Pi_{m perp} grad F
 * (Eqs. nablaLF, proj). */
int mm_gradient(mm_ctx* ctx, const double* m, const mm_params* p,
                double* grad_out, int projected);

/* Scalar potential of the last evaluation, [n_nodes] (0 on the outer
 * surface), internal units (Mref * 1 nm). */
int mm_get_potential(mm_ctx* ctx, double* phi_out);

/* Truncated preconditioner solve of Eq. (precond) by Algorithm 1 with
 * li1-li3 (Sec. 2.2, 3.1) at the state of the last evaluation (mm_energy or
 * mm_gradient): y ~ H(m)^{-1} g for the projected gradient g there.
 * y_out [n_nodes][3]; *steps (may be NULL) = products with H.  With
 * p->precision = 1, the precision form's FP32 apply. */
int mm_precond_solve(mm_ctx* ctx, const mm_params* p, double* y_out,
                     int64_t* steps);

/* One product with the approximate Hessian of Eq. (precond) at the state of
 * the last evaluation: out = H(m) v, v and out [n_nodes][3] host arrays. */
int mm_hessian_apply(mm_ctx* ctx, const mm_params* p, const double* v,
                     double* out);

/* One product with the scalar-potential stiffness (Sec. 3.1):
 * out = K_phi v on the unknowns, with v and out [n_nodes] host arrays
 * (entries on the outer surface are ignored / written as 0). */
int mm_potential_matvec(mm_ctx* ctx, const double* v, double* out);

/* One product with an operator of Eq. (energy) (Sec. 2.2, 3.1), the same
 * device code the minimiser applies, in internal units (lengths in nm,
 * magnetisation in units of Mref; v and out are host arrays indexed by node):
 *   MM_OP_DIV    out[n_nodes]    = D v: the right-hand side of the potential
 *                equation K_phi phi = D m for v = m ([n_nodes][3], used as
 *                given, not normalised); 0 off the potential unknowns
 *   MM_OP_DIVT   out[n_nodes][3] = D^T v for a potential v [n_nodes] (entries
 *                on the outer surface ignored): the magnetostatic part of
 *                grad F; 0 on non-magnetic nodes
 *   MM_OP_LOCAL  out[n_nodes][3] = (C_A + C_K) v for v [n_nodes][3]: the
 *                exchange and anisotropy part of grad F
 * MM_ERR_ARG for an unknown op or null arrays. */
enum { MM_OP_DIV = 0, MM_OP_DIVT = 1, MM_OP_LOCAL = 2 };
int mm_operator_apply(mm_ctx* ctx, int32_t op, const double* v, double* out);

/* Demagnetisation curve (Sec. 3.1): for each of n_fields applied fields
 * mu0*H (tesla, [n_fields][3]) set the field and minimise from the previous
 * minimum.  stats_out [n_fields] (may be NULL).  Returns the first non-OK
 * status met, after running every field. */
int mm_demag_curve(mm_ctx* ctx, int64_t n_fields, const double* fields,
                   const mm_params* p, mm_stats* stats_out);

/* Coercive field of a demagnetisation curve (Sec. 3.1: the field is swept
 * in small steps and each step minimised from the previous minimum).  Host
 * only, no context.  The sweep direction is u = (fields[n-1] - fields[0]) /
 * its norm (or fields[n-1] / its norm when the two ends coincide); H_c is
 * |mu0 H . u| where M . u first changes sign, linearly interpolated between
 * the two bracketing steps (a step with M . u exactly 0 gives its own
 * field).
 *   fields [n][3] mu0*H in tesla, M [n][3] reduced magnetisation per step
 *   (mm_stats.M); *hc_out in tesla, *found = 1, or *found = 0 (and *hc_out
 *   untouched) when M . u never changes sign.
 * MM_ERR_ARG for null pointers, n < 2, non-finite input or a zero sweep
 * direction. */
int mm_coercive_field(int64_t n, const double* fields, const double* M, double* hc_out, int32_t* found);

/* Energy and gradient at m without any device allocation in the call.
 * The paper has no counterpart; this entry point is for callers that cannot
 * call cudaMalloc: a process whose device memory is handed in full to its
 * own pool allocator or held to a fixed quota, or a latency-bound loop that
 * cannot afford the device-wide synchronisation of cudaFree.  It runs the
 * same potential solve and energy/gradient pass as mm_energy and
 * mm_gradient, on the operators assembled by mm_upload_mesh (which did
 * allocate, once), at the field of the last mm_set_field, with every work
 * vector in one fixed 8 MiB device array of the library.  That array is
 * held by every GPU that loads the library until the process exits.
 *   m_dev      [n_nodes][3] doubles on the context's device (normalised here)
 *   grad_dev   [n_nodes][3] output, or NULL; projected = 1 gives Pi grad F;
 *              internal units as in mm_gradient; non-magnetic rows are 0
 *   energy_dev 5 doubles output: F and the four terms of mm_energy, in J
 * The potential solve runs in FP64 (the precision field of p is ignored)
 * and starts from zero on every call.  Size limit:
 * 11 n_mag + 6 n_phi doubles plus about 32 doubles per persistent block
 * must fit in 8 MiB (about n_phi <= 150,000 for a cube in a box twice its
 * size); larger problems return MM_ERR_ARG with the required size.  Every
 * call looks up the array's device address on the context's device
 * (cudaGetSymbolAddress, with that device current; a device reset thus
 * needs no special handling): make the first call on a device before any
 * stream capture.  A zero or non-finite vector of m_dev on a magnetic node
 * returns MM_ERR_NONFINITE.  Every call shares the array and leaves its
 * contents behind; calls that overlap on the GPU (other contexts or threads
 * on the same device) race on it.  Synchronises the context's stream. */
int mm_energy_gradient_noalloc(mm_ctx* ctx, const double* m_dev, const mm_params* p,
                               double* grad_dev, int projected, double* energy_dev);

/* ---- Batched minimisation (no counterpart in the paper: many independent
 * magnets, e.g. sensor elements of different shapes, solved together).
 * A batch groups contexts on one device, each with an uploaded mesh.  One
 * cooperative launch runs Algorithm 4 for every member, each on its own team
 * of blocks (teams synchronise only internally, so members of different
 * sizes and iteration counts proceed independently).  Members keep their
 * own state (m, potential, field); after a batch call the member contexts
 * can be read with mm_get_magnetization etc.  At most as many members as
 * co-resident blocks (about 3 x the SM count). */
typedef struct mm_batch mm_batch;

/* Split total_blocks over n teams in proportion to work[t]^gamma, at least
 * one block each (largest-remainder rounding).  Pure host function. */
int mm_batch_plan(int n, const int64_t* work, int total_blocks, double gamma,
                  int32_t* blocks_out);
int mm_batch_create(mm_batch** b, int n, mm_ctx* const* ctxs);
void mm_batch_destroy(mm_batch* b);
const char* mm_batch_last_error(const mm_batch* b);
/* Kernel instantiation (2, 3 or 4 blocks per SM) and team-split exponent. */
int mm_batch_config(mm_batch* b, int blocks_per_sm, double gamma);
/* Minimise every member at its current field from its current m (one
 * launch); stats_out [n] (may be NULL).  Returns the first non-OK status. */
int mm_batch_minimize(mm_batch* b, const mm_params* p, mm_stats* stats_out);
/* Demagnetisation curves of every member: fields [n_steps][n][3] (mu0*H, T).
 * One field step (set the fields, solve every member, record the stats) is
 * captured once as a CUDA graph and replayed n_steps times with no host
 * round trip in between.  stats_out [n_steps][n] (may be NULL). */
int mm_batch_demag_curve(mm_batch* b, int64_t n_steps, const double* fields,
                         const mm_params* p, mm_stats* stats_out);
/* Tile shape of every member in batch launches, as in mm_set_tiles (the
 * members' own settings are not used by batch launches). */
int mm_batch_set_tiles(mm_batch* b, int32_t rows_per_thread, int32_t restrict_lanes);
/* The configuration batch launches use: kernel instantiation, team-split
 * exponent, rows per thread and restriction lanes (defaults resolved).
 * Any output may be NULL. */
int mm_batch_get_config(const mm_batch* b, int32_t* blocks_per_sm, double* gamma,
                        int32_t* rows_per_thread, int32_t* restrict_lanes);
/* Time configurations on a short minimisation (max_iter capped at 25) of
 * the members' current states, restoring the states after each trial, and
 * keep the fastest: first the 3 kernel instantiations x 3 team-split
 * exponents (0.5, 0.75, 1) at the default tile shape, then at the best of
 * those the 6 tile shapes (rows per thread 2 or 1 x restriction lanes 8, 4
 * or 16).  The chosen tile shape is read with mm_batch_get_config. */
int mm_batch_autotune(mm_batch* b, const mm_params* p, int* chosen_blocks_per_sm,
                      double* chosen_gamma, double* best_ms);
/* Device time (ms) of the last batch launch or curve. */
int mm_batch_last_ms(mm_batch* b, double* ms);

/* ---- Learned warm start (no counterpart in the paper).  A per-node
 * multilayer perceptron 16 -> 128 -> 128 -> 128 -> 4 (ReLU) maps local
 * features of a converged state and the next field increment to a
 * correction of m and of the scalar potential; Algorithm 4 then runs to
 * t1-t3 from the corrected state as usual, so the network only moves the
 * starting point.  Forward and backward passes run on the tensor cores
 * (BF16 operands, FP32 accumulation); FP32 master weights and Adam.
 * Parameters (floats): W1 [128][16], b1, W2 [128][128], b2, W3, b3,
 * W4 [4][128], b4, weights row-major [out][in]. */
typedef struct mm_mlp mm_mlp;
int64_t mm_mlp_param_count(void);
/* He-uniform initial weights from a seeded generator, zero biases. */
int mm_mlp_create(mm_mlp** mlp, int device, uint64_t seed);
void mm_mlp_destroy(mm_mlp* mlp);
int mm_mlp_set_params(mm_mlp* mlp, const float* params, int64_t count);
/* Tensor-core path of the forward pass and of the weight gradients: 0
 * (default) = tcgen05 MMAs with FP32 accumulators in tensor memory (M = 128
 * per MMA), 1 = the warp-level mma.sync path, kept as a measured
 * comparison.  Both round at the same points (BF16 inputs, weights and
 * hidden activations; FP32 accumulation).  A tensor-core wait that runs out (2 s) makes the next
 * synchronising MLP call return MM_ERR_DEVICE_TIMEOUT. */
int mm_mlp_set_tensor_path(mm_mlp* mlp, int path);
int mm_mlp_get_params(mm_mlp* mlp, float* params, int64_t count);
/* Input standardisation applied in FP32 before the BF16 first layer:
 * x_c <- (x_c - mean[c]) / std[c] (default mean 0, std 1). */
int mm_mlp_set_input_norm(mm_mlp* mlp, const float mean[16], const float stdev[16]);
/* Y_dev [n][4] = network(X_dev [n][16]) (device arrays); synchronises. */
int mm_mlp_forward(mm_mlp* mlp, const float* X_dev, int64_t n, float* Y_dev);
/* Mean squared error over all outputs against T_dev [n][4] and its gradient
 * (host array in the parameter layout, may be NULL); no update. */
int mm_mlp_gradient(mm_mlp* mlp, const float* X_dev, const float* T_dev, int64_t n,
                    float* grad_host, float* loss_out);
/* One Adam step (beta 0.9 / 0.999) on the mean squared error; loss_out may
 * be NULL (then no synchronisation). */
int mm_mlp_train_step(mm_mlp* mlp, const float* X_dev, const float* T_dev, int64_t n,
                      float lr, float* loss_out);
/* Set the input standardisation from data: per feature, the mean and the
 * unbiased standard deviation of X_dev [n][16] (device, FP64 sums, blocks
 * in a fixed order); a feature whose deviation is below 1e-6 (|mean| + 1)
 * is only centred.  n >= 2.  mm_mlp_get_input_norm reads back the mean and
 * 1/std in use. */
int mm_mlp_fit_input_norm(mm_mlp* mlp, const float* X_dev, int64_t n);
int mm_mlp_get_input_norm(mm_mlp* mlp, float mean[16], float inv_stdev[16]);
/* Target scales for training: *scale_m = the unbiased standard deviation of
 * the m-columns T[:, 0:3] taken together, *scale_phi that of T[:, 3] (each
 * at least 1e-12), and Tn_dev [n][4] = T_dev with those columns divided by
 * them (device arrays; Tn_dev may be T_dev).  n >= 2. */
int mm_mlp_fit_target_scales(mm_mlp* mlp, const float* T_dev, int64_t n, float* Tn_dev, double* scale_m,
                             double* scale_phi);
/* Training targets of one field step from the features of the converged
 * states before (X0_dev) and after (X1_dev) it, both [n][16] from
 * mm_warmstart_features for the same step: T_dev [n][4] = (m_after -
 * m_before, phi_after - phi_before) / |dh|, |dh| the norm of the field
 * increment (features 12..14, internal units).  *dh_out = |dh| (0: T_dev
 * left untouched); *max_change_out = the largest nodal |m_after - m_before|
 * (a switching step shows as a large value). */
int mm_warmstart_targets(mm_mlp* mlp, const float* X0_dev, const float* X1_dev, int64_t n, float* T_dev,
                         double* dh_out, double* max_change_out);
/* Features of every magnetic node of the context's current state for the
 * step to the applied field mu0h_next (tesla): m, effective field, exchange
 * field, anisotropy field (fields per unit Ms weight, internal units), the
 * field increment (internal units) and the scalar potential at the node.
 * X_dev [n_mag][16] floats, magnetic nodes in ascending node id. */
int mm_warmstart_features(mm_ctx* ctx, const double mu0h_next[3], float* X_dev);
/* Predict and apply the warm start for the step to mu0h_next:
 * m_i <- N(m_i + c scale_m |dh| y_i[0:3]), phi_i += c scale_phi |dh| y_i[3] on
 * the magnetic nodes (|dh| = norm of the field increment in internal
 * units), c = min(1, max_change / max_i |predicted change of m_i|) when
 * max_change > 0 (a cap that keeps the prediction from carrying the state
 * over a small energy barrier; the minimiser must follow the local minimum).
 * Then set the field and call mm_minimize as usual. */
int mm_warmstart_apply(mm_ctx* ctx, mm_mlp* mlp, const double mu0h_next[3],
                       double scale_m, double scale_phi, double max_change);

/* j_max autotuning (Tables 1, 3 and 4 of the paper choose j_max per problem
 * class by the time to solution): from the current state, minimise the
 * n_fields applied fields mu0*H (tesla, [n_fields][3]) in turn with p's
 * parameters and each candidate j_max (candidates [n_candidates], >= 0),
 * timing the solver launches with CUDA events, and restore the state (m,
 * potential, applied field) after each trial.  *best_jmax = the fastest
 * candidate; ms_out [n_candidates] (may be NULL) = each candidate's device
 * time.  The state is left as it was on entry.  Synchronises. */
int mm_autotune_jmax(mm_ctx* ctx, const mm_params* p, int64_t n_fields, const double* fields,
                     const int32_t* candidates, int32_t n_candidates, int32_t* best_jmax, double* ms_out);

/* Device time (ms) of the last persistent-kernel launch, from CUDA events
 * on the context's stream; synchronises. */
int mm_last_kernel_ms(mm_ctx* ctx, double* ms);

/* The stream the context runs on (a cudaStream_t). */
void* mm_stream(const mm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MMNCG_H */
