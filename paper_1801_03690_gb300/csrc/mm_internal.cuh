// Internal data structures of the mmncg library (host and device).
//
// Layout in HBM (all FP64 unless stated):
//   * magnetic nodes i in [0, nm): m, gradients, directions and the inner
//     solve vectors are SoA 3-vectors, component c of node i at v[c*nm + i];
//   * potential unknowns p in [0, nphi): the first nm are the magnetic nodes
//     (same order), the rest are the air nodes off the outer surface.  A
//     magnetic node on the outer surface keeps an identity row (phi = 0);
//   * both sparse graphs are SELL-32: rows in slices of 32, each slice
//     column-major with the slice's max row length, entry (row r, k) at
//     sptr[r/32] + 32*k + r%32; padding entries point at their own row with
//     value 0.  One warp reads one slice: every load of col/val is a single
//     coalesced 128/256-byte transaction.
#pragma once
#include <cstdint>

#define MM_BLOCK 256
#define MM_SELL 32
#define MM_MAXRED 16          // reduction values per phase
#define MM_NSLOT 3            // state slots: current, trial t, trial s
#define MM_MAXLEV 6           // smoothed levels of the potential preconditioner

namespace mm {

enum Mode : int {
    MODE_MINIMIZE = 0,
    MODE_EVAL = 1,
    MODE_PRECOND = 2,
    MODE_HESS = 3,
    MODE_KPHI = 4,
    MODE_DIV = 5,
    MODE_DIVT = 6,
    MODE_LOCAL = 7,
};

enum DevStatus : int {
    ST_RUNNING = -100,
    ST_OK = 0,
    ST_NOT_CONVERGED = 1,
    ST_STALLED = 2,
    ST_NONFINITE = -5,
    ST_TIMEOUT = -6,
};

struct Params {
    double tau_F;
    int jmax;
    int max_iter;
    double theta_max;
    double c1;
    int max_backtrack;
    int keep_last_term;
    double poisson_tol;
    int poisson_max_iter;
    int precision;           // 0 = FP64, 1 = FP32 potential solve + FP64 refinement
    int amg;                 // 1 = aggregation multigrid preconditioner in the FP32 solve
    double inner_tol;        // FP32 solve: relative residual reduction per refinement
    int max_refine;          // FP64 refinement steps per potential solve
    int beta_rule;           // 0 = beta*ZA, 1 = beta*FR, 2 = beta*PRP
    int poisson_sched;       // 1 = potential tolerance tied to t1
    double poisson_tol_max;  // loosest scheduled potential tolerance
};

// Scalars written back by the kernel (block 0) and read by the host.
struct DevState {
    int cur;                 // index of the current slot
    int status;
    long long evals, nli, li, mi, ls_extra, mr;
    long long li2, li2_first, restarts, steepest;   // branch counters (mm_stats)
    double F;                // internal units
    double terms[4];         // exchange, anisotropy, demag, Zeeman (internal)
    double M[3];             // weighted mean magnetisation of the current slot
    double gmax;             // |g|_inf of the current slot
    double h[3];             // reduced applied field
    int y_is_g;              // 1 if the last preconditioner output is g itself
    int pad;
};

// Level l of the smoothed-aggregation multigrid preconditioner of the FP32
// potential solve (level 0: K_phi itself; level l+1: the Galerkin operator
// P^T A_l P of the smoothed prolongation P of the aggregates of level l).
// With x = omega D^-1 b (one damped-Jacobi step from zero), the V-cycle is
//   down: rpre = b - A x,   b_{l+1} = P^T rpre
//   up:   y = omega D^-1 (b + rpre) + U y_{l+1}
// with U = P - omega D^-1 A P, i.e. pre-smoothing, restriction of the
// residual, coarse correction and post-smoothing with the same damped
// Jacobi step: a symmetric operator (P^T rpre = U^T b).  Operators are
// FP32, SELL-32 except P^T (CSR).
// Entry 0 of a slice offset table that marks a slice with a column array.
#define MM_NO_TAB (-2147483647 - 1)

struct Level {
    int n;                   // rows of this level
    int nc;                  // rows of the next coarser level
    float omega;             // Jacobi damping of this level's smoother
    int wide;                // 1: P^T rows average over 160 entries (a warp per row)
    const long long* sptr;   // A_l (level 0: the FP32 copy of K_phi)
    const int* col;
    const float* val;
    const int* tab;          // level 0: the slice offset tables of K_phi (k_tab)
    const long long* u_sptr; // U (n rows, nc columns)
    const int* u_col;
    const float* u_val;
    const long long* t_ptr;  // P^T (nc rows, n columns) in CSR: its rows are wide
    const int* t_col;        // (the support of a smoothed aggregate), one warp
    const float* t_val;      // takes one row
    const float* dinv;       // 1 / diag(A_l)
    float* b;                // right-hand side (level 0: unused, the FP32 residual)
    float* x;                // omega D^-1 b (level 0: unused, amg_x0)
    float* rpre;             // b - A x
    float* y;                // output (level 0: the preconditioned residual)
};

struct Problem {
    int nm;                  // magnetic nodes
    int nphi;                // potential unknowns
    // magnetic graph (SELL-32): exchange stiffness K_A, and the divergence
    // coupling in both orientations: G(i, j) = D_{j i} (for D^T phi, row i a
    // magnetic node, column j a potential unknown) and B(j, i) = D_{j i}
    // (for D m, row j, column i); SoA by component, stride nnzm.
    const long long* m_sptr;
    const int* m_col;
    long long nnzm;
    const double* KA;
    const double* G;
    const double* B;
    const double* CK;        // [6][nm]: xx, xy, xz, yy, yz, zz of C_K blocks
    const double* w;         // [nm] lumped Ms weights
    const double* dinvA;     // [nm] 1 / diag(C_A) (1 where zero)
    // potential graph (SELL-32)
    const long long* p_sptr;
    const int* p_col;
    const double* Kp;
    const double* dinvP;     // [nphi] 1 / diag(K_phi)
    // state slots
    double* X[MM_NSLOT];     // [3][nm] unit vectors
    double* GR[MM_NSLOT];    // [3][nm] grad F
    double* GP[MM_NSLOT];    // [3][nm] projected gradient
    double* LAM[MM_NSLOT];   // [nm] lambda = m . grad F
    double* unorm;           // [nm] |x + a d| of the last trial point
    double* d;               // [3][nm] NCG direction
    // inner solve (Algorithm 1 on H)
    double* isol;            // [3][nm]
    double* ires;            // [3][nm] residual
    double* iprec;           // [3][nm] Jacobi-preconditioned residual
    double* idir[2];         // [3][nm] direction (double buffer)
    double* ihd;             // [3][nm] H * direction
    // precision form: the inner solve's H products and vectors in FP32
    // (isol stays FP64: the search direction is built from it)
    const float* KA32;       // [nnzm] K_A on the magnetic graph's SELL-32
    const float* CK32;       // [6][nm]
    const float* dinvA32;    // [nm]
    float* ires32;           // [3][nm]
    float* iprec32;          // [3][nm]
    float* idir32;           // [3][nm]
    float* ihd32;            // [3][nm]
    // potential solve (Algorithm 1 on K_phi)
    double* phi;             // [nphi] working potential (the last solve)
    double* PHI[MM_NSLOT];   // [nphi] potential of each state slot
    double* rhs;             // [nm] D m on the magnetic rows (zero elsewhere)
    double* pres;            // [nphi] residual
    double* pprec;           // [nphi] Jacobi-preconditioned residual
    double* pdir[2];         // [nphi] direction (double buffer)
    double* pq;              // [nphi] K_phi * direction
    // precision form: FP32 copies of K_phi and diag^-1, FP32 work vectors.
    // The FP32 K_phi has a SELL-32 layout of its own (k_sptr, k_col) with a
    // table of 8 column offsets per slice (k_tab): in a slice whose table
    // does not start with MM_NO_TAB, entry k of row r is column r + tab[k]
    // and k_col is not read (lattice stencils); other slices use k_col.
    const long long* k_sptr;
    const int* k_col;
    const int* k_tab;        // [slices][8], 32-byte aligned rows
    const float* Kp32;
    const float* dinvP32;
    float* pres32;           // [nphi] residual of the correction equation
    float* pprec32;
    float* pdir32;
    float* pq32;
    float* pdelta32;         // [nphi] correction
    // smoothed-aggregation multigrid (precision form)
    int nlev;                // smoothed levels (0: no hierarchy)
    int nco;                 // rows of the coarsest level (solved densely)
    Level lev[MM_MAXLEV];
    float* amg_x0;           // [nphi] omega D^-1 r of the FP32 residual r
    const float* ainv;       // [nco][nco] inverse of the coarsest operator
    float* bco;              // [nco] coarsest right-hand side
    float* yco;              // [nco] coarsest solution
    float amg_omega;         // Jacobi damping of the level-0 smoother
    // team machinery
    double* partials;        // [2][MM_MAXRED][nblocks]
    unsigned* bar;           // [0..1] = 64-bit arrival counter of the team barrier
    int* err;                // device error flag
    DevState* state;
    Params prm;
    int mode;
    // tile shape of the level-0 FP32 products and of the restrictions
    // (zero-initialised = the defaults): tile_rows 1 = one row per thread,
    // else two; restrict_lanes 4 or 16 lanes per coarse row, else 8 (levels
    // with wide rows always take a whole warp)
    int tile_rows;
    int restrict_lanes;
};

// Read-only view of a context for entry points defined outside mm_api.cu.
struct CtxView {
    const Problem* P;
    void* stream;                // cudaStream_t
    int device;
    int blocks;
    long long n_nodes;
    int nm, nphi;
    double Mref;
    double field_T[3];
    const int* mag_nodes;        // device
    const int* node_of_phi;      // device
    const unsigned char* ident;  // device
    bool has_mesh;
    const void* kernel;          // the solver kernel the context launches
    DevState* d_state;           // device
    long long nnz_mag, nnz_phi;  // true nonzeros of the two graphs
};

}  // namespace mm

struct mm_ctx;
namespace mm {
// Device function pointer of the solver kernel built for at least
// min_blocks resident blocks per SM (2, 3 or 4; others -> 3).
const void* solver_kernel(int min_blocks);
// The batched solver kernel (teams of blocks, one problem per team);
// min_blocks 3 or 4 (others -> 3).
const void* solver_batch_kernel(int min_blocks);
__attribute__((visibility("hidden"))) int ctx_view(mm_ctx* ctx, CtxView* out);
__attribute__((visibility("hidden"))) int ctx_fail(mm_ctx* ctx, int code, const char* msg);
// Copy the context's device state to its host mirror after work launched
// elsewhere (a batch) and mark the current state as evaluated.
__attribute__((visibility("hidden"))) int ctx_refresh_state(mm_ctx* ctx);
}  // namespace mm
