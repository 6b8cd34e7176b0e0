// C-ABI of the mmncg library (declared in include/mmncg.h): context,
// mesh upload (host-side graph construction, GPU assembly), state transfer
// and the launches of the persistent solver kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mmncg.h"
#include "mm_assemble.cuh"
#include "mm_internal.cuh"


namespace {

constexpr double kMu0 = 4e-7 * 3.14159265358979323846;

// ------------------------------------------------------------ small kernels

__global__ void k_set_m(int nm, const int* mag_nodes, const double* m_nodes, double* X, int* bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    const long long n = mag_nodes[i];
    const double a = m_nodes[3 * n], b = m_nodes[3 * n + 1], c = m_nodes[3 * n + 2];
    const double r = sqrt(a * a + b * b + c * c);
    if (!(r > 0.0) || !isfinite(r)) {
        atomicExch(bad, 1);
        X[i] = 0.0;
        X[nm + i] = 0.0;
        X[2 * nm + i] = 1.0;
        return;
    }
    X[i] = a / r;
    X[nm + i] = b / r;
    X[2 * nm + i] = c / r;
}

// out[node][3] = v[c*nm + i] for magnetic nodes (other rows untouched)
__global__ void k_scatter3(int nm, const int* mag_nodes, const double* v, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    const long long n = mag_nodes[i];
    out[3 * n] = v[i];
    out[3 * n + 1] = v[nm + i];
    out[3 * n + 2] = v[2 * nm + i];
}

__global__ void k_gather3(int nm, const int* mag_nodes, const double* in, double* v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    const long long n = mag_nodes[i];
    v[i] = in[3 * n];
    v[nm + i] = in[3 * n + 1];
    v[2 * nm + i] = in[3 * n + 2];
}

__global__ void k_scatter1(int np, const int* node_of_phi, const unsigned char* ident, const double* v,
                           double* out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    out[node_of_phi[p]] = ident[p] ? 0.0 : v[p];
}

__global__ void k_gather1(int np, const int* node_of_phi, const unsigned char* ident, const double* in,
                          double* v) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    v[p] = ident[p] ? 0.0 : in[node_of_phi[p]];
}

__global__ void k_set_field(mm::DevState* st, double h0, double h1, double h2) {
    st->h[0] = h0;
    st->h[1] = h1;
    st->h[2] = h2;
}

__global__ void k_set_cur(mm::DevState* st, int cur) { st->cur = cur; }

__global__ void k_to_f32(long long n, const double* a, float* b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

inline int nblk(long long n, int b = 256) { return (int)((n + b - 1) / b); }

}  // namespace

struct mm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nsm = 0;
    int blocks = 0;
    int blocks_per_sm_req = 0;
    const void* kernel = nullptr;
    std::string err;
    // mesh
    bool has_mesh = false;
    bool has_eval = false;
    int64_t n_nodes = 0;
    int nm = 0, nphi = 0;
    long long nnzm = 0, nnzp = 0;         // padded SELL entries
    long long nnzm_true = 0, nnzp_true = 0;
    std::vector<long long> amg_nnz_a, amg_nnz_u, amg_nnz_p;   // per multigrid level (host copy)
    double Mref = 0.0;
    double field_T[3] = {0, 0, 0};
    std::vector<void*> allocs;            // device buffers of the mesh
    mm::Problem P{};
    int tile_rows = 0, restrict_lanes = 0;   // mm_set_tiles (0 = default); kept across uploads
    long long k32_slices = 0, k32_table_slices = 0, k32_bytes = 0;   // FP32 K_phi layout
    mm::DevState* d_state = nullptr;      // device
    mm::DevState* h_state = nullptr;      // pinned host
    int* d_mag_nodes = nullptr;
    int* d_node_of_phi = nullptr;
    unsigned char* d_ident = nullptr;
    double* d_stage = nullptr;            // [n_nodes][3] staging
    int* d_flag = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
};

namespace {

int fail(mm_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail(ctx, MM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
int dalloc(mm_ctx* ctx, T** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, MM_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    }
    ctx->allocs.push_back(q);
    *p = (T*)q;
    return MM_OK;
}

// Free one device buffer of the mesh (allocated by dalloc).
void dfree(mm_ctx* ctx, const void* p) {
    for (size_t k = 0; k < ctx->allocs.size(); ++k)
        if (ctx->allocs[k] == p) {
            cudaFree(ctx->allocs[k]);
            ctx->allocs.erase(ctx->allocs.begin() + k);
            return;
        }
}

void free_mesh(mm_ctx* ctx) {
    for (void* p : ctx->allocs) cudaFree(p);
    ctx->allocs.clear();
    ctx->P = mm::Problem{};
    ctx->P.tile_rows = ctx->tile_rows;
    ctx->P.restrict_lanes = ctx->restrict_lanes;
    ctx->has_mesh = false;
    ctx->has_eval = false;
}

mm::Params to_params(const mm_params* p) {
    mm_params d;
    mm_default_params(&d);
    if (!p) p = &d;
    mm::Params q;
    q.tau_F = p->tau_F;
    q.jmax = p->jmax;
    q.max_iter = p->max_iter;
    q.theta_max = p->theta_max;
    q.c1 = p->c1;
    q.max_backtrack = p->max_backtrack;
    q.keep_last_term = p->keep_last_term;
    q.poisson_tol = p->poisson_tol;
    q.poisson_max_iter = p->poisson_max_iter;
    q.precision = p->precision;
    q.amg = p->amg;
    q.inner_tol = p->inner_tol;
    q.max_refine = p->max_refine;
    q.beta_rule = p->beta_rule;
    q.poisson_sched = p->poisson_sched;
    q.poisson_tol_max = p->poisson_tol_max;
    return q;
}

int check_params(mm_ctx* ctx, const mm_params* p) {
    if (!p) return MM_OK;
    if (!(p->tau_F > 0.0) || !(p->tau_F < 1.0)) return fail(ctx, MM_ERR_ARG, "tau_F must be in (0, 1)");
    if (p->jmax < 0) return fail(ctx, MM_ERR_ARG, "jmax must be >= 0");
    if (p->max_iter < 0) return fail(ctx, MM_ERR_ARG, "max_iter must be >= 0");
    if (!(p->theta_max > 0.0)) return fail(ctx, MM_ERR_ARG, "theta_max must be > 0");
    if (!(p->c1 > 0.0 && p->c1 < 1.0)) return fail(ctx, MM_ERR_ARG, "c1 must be in (0, 1)");
    if (p->max_backtrack < 0) return fail(ctx, MM_ERR_ARG, "max_backtrack must be >= 0");
    if (!(p->poisson_tol > 0.0)) return fail(ctx, MM_ERR_ARG, "poisson_tol must be > 0");
    if (p->poisson_max_iter < 1) return fail(ctx, MM_ERR_ARG, "poisson_max_iter must be >= 1");
    if (p->precision != 0 && p->precision != 1) return fail(ctx, MM_ERR_ARG, "precision must be 0 or 1");
    if (p->precision == 1 && !(p->inner_tol > 0.0 && p->inner_tol < 1.0))
        return fail(ctx, MM_ERR_ARG, "inner_tol must be in (0, 1)");
    if (p->precision == 1 && p->max_refine < 1) return fail(ctx, MM_ERR_ARG, "max_refine must be >= 1");
    if (p->amg != 0 && p->amg != 1) return fail(ctx, MM_ERR_ARG, "amg must be 0 or 1");
    if (p->beta_rule < 0 || p->beta_rule > 2) return fail(ctx, MM_ERR_ARG, "beta_rule must be 0, 1 or 2");
    if (p->poisson_sched != 0 && p->poisson_sched != 1) return fail(ctx, MM_ERR_ARG, "poisson_sched must be 0 or 1");
    if (p->poisson_sched && !(p->poisson_tol_max >= p->poisson_tol && p->poisson_tol_max < 1.0))
        return fail(ctx, MM_ERR_ARG, "poisson_tol_max must be in [poisson_tol, 1)");
    return MM_OK;
}

// Build SELL-32 slice pointers and columns from row adjacency lists.
void build_sell(const std::vector<std::vector<int>>& rows, std::vector<long long>& sptr,
                std::vector<int>& col, long long& nnz_true) {
    const long long n = (long long)rows.size();
    const long long ns = (n + 31) / 32;
    sptr.assign(ns + 1, 0);
    nnz_true = 0;
    for (long long s = 0; s < ns; ++s) {
        size_t w = 0;
        for (long long r = s * 32; r < std::min(n, s * 32 + 32); ++r) w = std::max(w, rows[r].size());
        sptr[s + 1] = sptr[s] + 32ll * (long long)w;
    }
    col.assign(sptr[ns], 0);
    for (long long s = 0; s < ns; ++s) {
        const long long w = (sptr[s + 1] - sptr[s]) / 32;
        for (int l = 0; l < 32; ++l) {
            const long long r = s * 32 + l;
            for (long long k = 0; k < w; ++k) {
                int c;
                if (r < n && k < (long long)rows[r].size()) {
                    c = rows[r][k];
                    ++nnz_true;
                } else {
                    c = (r < n) ? (int)r : 0;          // padding: own row, value 0
                }
                col[sptr[s] + 32 * k + l] = c;
            }
        }
    }
}

// CSR matrix on the host.
struct HostCsr {
    int n = 0;                  // rows
    int m = 0;                  // columns
    std::vector<long long> ptr;
    std::vector<int> col;
    std::vector<double> val;
};

// Greedy aggregation of the matrix graph (every stored entry is an edge,
// whatever its value): (1) a node whose neighbours are all free starts an
// aggregate with them; (2) remaining nodes join the aggregate of their
// first aggregated neighbour; (3) the rest become singletons.  Returns the
// number of aggregates.
int aggregate(const HostCsr& A, std::vector<int>& agg) {
    const int n = A.n;
    agg.assign(n, -1);
    int na = 0;
    for (int i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        bool free_nb = true;
        for (long long e = A.ptr[i]; e < A.ptr[i + 1] && free_nb; ++e)
            if (A.col[e] != i && agg[A.col[e]] >= 0) free_nb = false;
        if (!free_nb) continue;
        agg[i] = na;
        for (long long e = A.ptr[i]; e < A.ptr[i + 1]; ++e) agg[A.col[e]] = na;
        ++na;
    }
    std::vector<int> first(agg);
    for (int i = 0; i < n; ++i) {
        if (first[i] >= 0) continue;
        for (long long e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
            const int j = A.col[e];
            if (j != i && first[j] >= 0) {
                agg[i] = first[j];
                break;
            }
        }
    }
    for (int i = 0; i < n; ++i)
        if (agg[i] < 0) agg[i] = na++;
    return na;
}

// C = A B (sparse, dense accumulator over the columns of B; entries that
// cancel exactly are kept, columns in first-touch order).
HostCsr spgemm(const HostCsr& A, const HostCsr& B) {
    HostCsr C;
    C.n = A.n;
    C.m = B.m;
    C.ptr.assign(A.n + 1, 0);
    std::vector<double> acc(B.m, 0.0);
    std::vector<int> mark(B.m, -1), cols;
    for (int i = 0; i < A.n; ++i) {
        cols.clear();
        for (long long e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
            const int k = A.col[e];
            const double a = A.val[e];
            for (long long f = B.ptr[k]; f < B.ptr[k + 1]; ++f) {
                const int j = B.col[f];
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0.0;
                    cols.push_back(j);
                }
                acc[j] += a * B.val[f];
            }
        }
        for (int j : cols) {
            C.col.push_back(j);
            C.val.push_back(acc[j]);
        }
        C.ptr[i + 1] = (long long)C.col.size();
    }
    return C;
}

HostCsr transpose(const HostCsr& A) {
    HostCsr T;
    T.n = A.m;
    T.m = A.n;
    T.ptr.assign(A.m + 1, 0);
    for (int c : A.col) T.ptr[c + 1]++;
    for (int j = 0; j < A.m; ++j) T.ptr[j + 1] += T.ptr[j];
    T.col.resize(A.col.size());
    T.val.resize(A.val.size());
    std::vector<long long> fill(T.ptr.begin(), T.ptr.end() - 1);
    for (int i = 0; i < A.n; ++i)
        for (long long e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
            const long long f = fill[A.col[e]]++;
            T.col[f] = i;
            T.val[f] = A.val[e];
        }
    return T;
}

// B - s D A for a diagonal D (row scaling), B and A of the same shape.
HostCsr minus_scaled_rows(const HostCsr& B, double s, const std::vector<double>& D, const HostCsr& A) {
    HostCsr C;
    C.n = B.n;
    C.m = B.m;
    C.ptr.assign(B.n + 1, 0);
    std::vector<double> acc(B.m, 0.0);
    std::vector<int> mark(B.m, -1), cols;
    for (int i = 0; i < B.n; ++i) {
        cols.clear();
        auto add = [&](int j, double v) {
            if (mark[j] != i) {
                mark[j] = i;
                acc[j] = 0.0;
                cols.push_back(j);
            }
            acc[j] += v;
        };
        for (long long e = B.ptr[i]; e < B.ptr[i + 1]; ++e) add(B.col[e], B.val[e]);
        for (long long e = A.ptr[i]; e < A.ptr[i + 1]; ++e) add(A.col[e], -s * D[i] * A.val[e]);
        for (int j : cols) {
            C.col.push_back(j);
            C.val.push_back(acc[j]);
        }
        C.ptr[i + 1] = (long long)C.col.size();
    }
    return C;
}

// SELL-32 layout of a host CSR (values converted to V); padding entries
// carry value 0 and their own row as column where that is a column of A,
// else 0.
template <class V>
void csr_to_sell(const HostCsr& A, std::vector<long long>& sptr, std::vector<int>& col, std::vector<V>& val) {
    const long long n = A.n, ns = (n + 31) / 32;
    sptr.assign(ns + 1, 0);
    for (long long s = 0; s < ns; ++s) {
        long long w = 0;
        for (long long r = s * 32; r < std::min(n, s * 32 + 32); ++r) w = std::max(w, A.ptr[r + 1] - A.ptr[r]);
        sptr[s + 1] = sptr[s] + 32 * w;
    }
    col.assign(sptr[ns], 0);
    val.assign(sptr[ns], V(0));
    for (long long s = 0; s < ns; ++s) {
        const long long w = (sptr[s + 1] - sptr[s]) / 32;
        for (int l = 0; l < 32; ++l) {
            const long long r = s * 32 + l;
            for (long long k = 0; k < w; ++k) {
                const long long e = sptr[s] + 32 * k + l;
                if (r < n && k < A.ptr[r + 1] - A.ptr[r]) {
                    col[e] = A.col[A.ptr[r] + k];
                    val[e] = (V)A.val[A.ptr[r] + k];
                } else {
                    col[e] = (r < A.m) ? (int)r : 0;   // padding: a valid column, value 0
                }
            }
        }
    }
}

// The FP32 copy of K_phi in SELL-32 with slice offset tables (the device
// reads it as Problem::k_sptr / k_col / k_tab / Kp32).  A slice whose rows
// couple, all together, to at most 8 distinct offsets c - r (on a
// rectilinear Kuhn lattice: the diagonal and the six axis neighbours), with
// r + offset a row of the matrix for every row r of the slice and every
// offset, gets those offsets in ascending order as its table; each of its
// rows stores one value per offset (0 where the row has no such coupling),
// so a product loads no columns there.  Rows are column-sorted (the output of
// prune_noise), so a table row lists the row's couplings in column order
// with zeros between them and its sums equal those of the plain layout.
// Other slices keep plain SELL-32 columns and MM_NO_TAB in table entry 0.
struct K32Layout {
    std::vector<long long> sptr;
    std::vector<int> col;
    std::vector<float> val;
    std::vector<int> tab;          // [slices][8]
    long long table_slices = 0;
    long long bytes = 0;           // matrix bytes one product loads
};

K32Layout k32_layout(const HostCsr& K) {
    K32Layout L;
    const long long n = K.n, ns = (n + 31) / 32;
    L.sptr.assign(ns + 1, 0);
    L.tab.assign(ns * 8, 0);
    std::vector<char> has_tab(ns, 0);
    std::vector<int> D;
    for (long long s = 0; s < ns; ++s) {
        const long long r0 = 32 * s, r1 = std::min(n, r0 + 32);
        long long wmax = 0;
        for (long long r = r0; r < r1; ++r) wmax = std::max(wmax, K.ptr[r + 1] - K.ptr[r]);
        bool ok = true;
        D.clear();
        for (long long r = r0; r < r1 && ok; ++r) {
            for (long long e = K.ptr[r]; e < K.ptr[r + 1]; ++e) {
                const int d = (int)(K.col[e] - r);
                if (std::find(D.begin(), D.end(), d) == D.end()) {
                    if (D.size() == 8) {
                        ok = false;
                        break;
                    }
                    D.push_back(d);
                }
            }
        }
        if (ok) {
            std::sort(D.begin(), D.end());
            for (long long r = r0; r < r1 && ok; ++r)
                for (int d : D)
                    if (r + d < 0 || r + d >= n) ok = false;
        }
        has_tab[s] = ok;
        const long long w = ok ? (long long)D.size() : wmax;
        L.sptr[s + 1] = L.sptr[s] + 32 * w;
        if (ok) {
            for (size_t k = 0; k < D.size(); ++k) L.tab[s * 8 + k] = D[k];
            ++L.table_slices;
            L.bytes += 4 * w * (r1 - r0) + 32;
        } else {
            L.tab[s * 8] = MM_NO_TAB;
            L.bytes += 8 * (K.ptr[r1] - K.ptr[r0]) + 32;
        }
    }
    L.col.assign(L.sptr[ns], 0);
    L.val.assign(L.sptr[ns], 0.0f);
    for (long long s = 0; s < ns; ++s) {
        const long long w = (L.sptr[s + 1] - L.sptr[s]) / 32;
        for (int l = 0; l < 32; ++l) {
            const long long r = 32 * s + l;
            const long long b = r < n ? K.ptr[r] : 0, e = r < n ? K.ptr[r + 1] : 0;
            long long q = b;
            for (long long k = 0; k < w; ++k) {
                const long long x = L.sptr[s] + 32 * k + l;
                if (r >= n) {
                    L.col[x] = 0;                            // past the last row: never read
                } else if (has_tab[s]) {
                    const long long c = r + L.tab[s * 8 + k];
                    L.col[x] = (int)c;
                    if (q < e && K.col[q] == c) L.val[x] = (float)K.val[q++];
                } else if (q < e) {
                    L.col[x] = K.col[q];
                    L.val[x] = (float)K.val[q++];
                } else {
                    L.col[x] = (int)r;                       // padding: column r, value 0
                }
            }
        }
    }
    return L;
}

// Entries that are zero in exact arithmetic but not in floating point.
// On a rectilinear (uniform or graded) Kuhn lattice the P1 Laplacian
// couples a node only to its six axis neighbours: the couplings along face
// and body diagonals are exactly zero, yet the assembled sums of b_i.b_j
// leave rounding residues of ~1e-17 relative to the diagonal.  They are
// dropped from the operators the potential solve applies; a coupling kept
// on a general mesh is above 1e-7 relative (jittered lattices), and dropping
// one below the threshold changes a product by less than 1e-12 relative.
constexpr double kNoiseRel = 1e-12;

// A without its off-diagonal entries a_ij with |a_ij| <= kNoiseRel *
// sqrt(|a_ii a_jj|) (square A), columns ascending within each row (the
// greedy aggregation breaks ties by storage order, so the order is fixed).
HostCsr prune_noise(const HostCsr& A) {
    std::vector<double> dg(A.n, 0.0);
    for (int i = 0; i < A.n; ++i)
        for (long long e = A.ptr[i]; e < A.ptr[i + 1]; ++e)
            if (A.col[e] == i) dg[i] = std::fabs(A.val[e]);
    HostCsr B;
    B.n = A.n;
    B.m = A.m;
    B.ptr.assign(A.n + 1, 0);
    B.col.reserve(A.col.size());
    B.val.reserve(A.val.size());
    std::vector<std::pair<int, double>> row;
    for (int i = 0; i < A.n; ++i) {
        row.clear();
        for (long long e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
            const int j = A.col[e];
            if (j != i && !(std::fabs(A.val[e]) > kNoiseRel * std::sqrt(dg[i] * dg[j]))) continue;
            row.emplace_back(j, A.val[e]);
        }
        std::sort(row.begin(), row.end(), [](const std::pair<int, double>& a, const std::pair<int, double>& b) {
            return a.first < b.first;
        });
        for (const auto& q : row) {
            B.col.push_back(q.first);
            B.val.push_back(q.second);
        }
        B.ptr[i + 1] = (long long)B.col.size();
    }
    return B;
}

// Inverse of a small SPD matrix, FP64, row-major:
// A = L L^T (Cholesky), L^-1 row by row, A^-1 = L^-T L^-1.  All inner loops
// run along rows.  Returns false if A is not numerically positive definite.
bool dense_inverse(const HostCsr& A, std::vector<double>& inv) {
    const int n = A.n;
    std::vector<double> L((size_t)n * n, 0.0), Li((size_t)n * n, 0.0), acc(n);
    for (int i = 0; i < n; ++i)
        for (long long e = A.ptr[i]; e < A.ptr[i + 1]; ++e) L[(size_t)i * n + A.col[e]] += A.val[e];
    for (int j = 0; j < n; ++j) {
        double* Lj = &L[(size_t)j * n];
        double d = Lj[j];
        for (int k = 0; k < j; ++k) d -= Lj[k] * Lj[k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        Lj[j] = d;
        for (int i = j + 1; i < n; ++i) {
            double* Lr = &L[(size_t)i * n];
            double v = Lr[j];
            for (int k = 0; k < j; ++k) v -= Lr[k] * Lj[k];
            Lr[j] = v / d;
        }
    }
    for (int i = 0; i < n; ++i) {                   // row i of L^-1
        const double* Lr = &L[(size_t)i * n];
        std::fill(acc.begin(), acc.begin() + i, 0.0);
        for (int k = 0; k < i; ++k) {
            const double c = Lr[k];
            const double* Lk = &Li[(size_t)k * n];
            for (int j = 0; j <= k; ++j) acc[j] += c * Lk[j];
        }
        double* out = &Li[(size_t)i * n];
        const double di = 1.0 / Lr[i];
        for (int j = 0; j < i; ++j) out[j] = -acc[j] * di;
        out[i] = di;
    }
    std::vector<double> X((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) {                   // X += row_k^T row_k
        const double* Lk = &Li[(size_t)k * n];
        for (int i = 0; i <= k; ++i) {
            const double c = Lk[i];
            double* Xi = &X[(size_t)i * n];
            for (int j = 0; j <= k; ++j) Xi[j] += c * Lk[j];
        }
    }
    inv.swap(X);
    return true;
}

template <class T>
int upload(mm_ctx* ctx, T** dst, const T* src, size_t count) {
    int rc = dalloc(ctx, dst, count);
    if (rc) return rc;
    if (count) CK_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return MM_OK;
}

// Upload a host CSR matrix in SELL-32 form with FP32 values.
int upload_sell(mm_ctx* ctx, const HostCsr& A, const long long** sptr, const int** col, const float** val) {
    std::vector<long long> sp;
    std::vector<int> c;
    std::vector<float> v;
    csr_to_sell(A, sp, c, v);
    long long* dsp;
    int* dc;
    float* dv;
    int rc;
    if ((rc = upload(ctx, &dsp, sp.data(), sp.size()))) return rc;
    if ((rc = upload(ctx, &dc, c.data(), c.size()))) return rc;
    if ((rc = upload(ctx, &dv, v.data(), v.size()))) return rc;
    *sptr = dsp;
    *col = dc;
    *val = dv;
    return 0;
}

constexpr int kCoarseDense = 1536;      // coarsest level solved by a dense inverse
constexpr double kAmgOmega = 0.9;       // Jacobi damping of the smoother, at most ...
constexpr double kAmgOmegaRho = 1.95;   // ... 1.95 / rho (rho >= the spectral radius of D^-1 A)

// Smoothed-aggregation multigrid hierarchy, built on the host in FP64 from
// level 0's CSR matrix A.  Level 0 aggregates on A's stored pattern (the
// mesh graph: values ignored, so rounding cannot change the aggregates) and
// computes with A without its rounding residues (prune_noise); every
// coarser level is the Galerkin operator without its residues, aggregated
// on its own pattern.  Per level: greedy aggregates, tentative
// prolongation P_t (piecewise constant), P = (I - w_p D^-1 A) P_t with
// w_p = 2 / rho, rho the Gershgorin bound of the spectral radius of D^-1 A,
// the Galerkin operator P^T A P, and the smoothed prolongation
// U = P - omega D^-1 A P used by the V-cycle with its transpose;
// omega = min(0.9, 1.95 / rho) keeps omega times the spectral radius below 2,
// so the damped-Jacobi smoother converges and the cycle is positive
// definite.  (A CPU scan on the hard-cube potential matrix put w_p in
// [1.3, 1.7] x 4 / (3 rho) and omega in [0.85, 0.95] on a plateau of about
// 20 V-cycle-preconditioned CG steps per 1e-6 residual reduction, against
// 23 with w_p = 4 / (3 rho), omega = 0.8.)
struct AmgHostLevel {
    double omega;
    HostCsr A, U, Pt;                    // Pt: the restriction P^T (CSR)
    std::vector<double> dinv;
};

struct AmgHost {
    std::vector<AmgHostLevel> lev;       // smoothed levels
    int nco = 0;                         // rows of the coarsest level
    long long nnz_co = 0;                // its nonzeros
    std::vector<double> ainv;            // [nco][nco] its inverse
};

// Returns false (no hierarchy: Jacobi only) when A is at most the dense
// size, the coarsening stalls before it, or the coarsest operator is not
// numerically positive definite.
bool build_amg_host(HostCsr A, AmgHost& H) {
    H = AmgHost();
    if (A.n <= kCoarseDense) return false;
    while ((int)H.lev.size() < MM_MAXLEV && A.n > kCoarseDense) {
        std::vector<int> agg;
        const int nc = aggregate(A, agg);                 // on the stored pattern
        if (nc > A.n / 2) break;                          // coarsening stalled
        if (H.lev.empty()) A = prune_noise(A);            // level 0: numerics without residues
        std::vector<double> dinv(A.n, 1.0);
        double rho = 0.0;
        for (int i = 0; i < A.n; ++i) {
            double d = 0.0, off = 0.0;
            for (long long e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
                if (A.col[e] == i) d = A.val[e];
                off += std::fabs(A.val[e]);
            }
            if (d > 0.0) {
                dinv[i] = 1.0 / d;
                rho = std::max(rho, off / d);
            }
        }
        HostCsr Pt;
        Pt.n = A.n;
        Pt.m = nc;
        Pt.ptr.resize(A.n + 1);
        Pt.col = agg;
        Pt.val.assign(A.n, 1.0);
        for (int i = 0; i <= A.n; ++i) Pt.ptr[i] = i;
        if (!(rho > 0.0)) rho = 2.0;
        HostCsr Pm = minus_scaled_rows(Pt, 2.0 / rho, dinv, spgemm(A, Pt));
        HostCsr AP = spgemm(A, Pm);
        HostCsr Cc = spgemm(transpose(Pm), AP);
        AmgHostLevel h;
        h.omega = std::min(kAmgOmega, kAmgOmegaRho / rho);
        h.U = minus_scaled_rows(Pm, h.omega, dinv, AP);
        h.Pt = transpose(Pm);
        h.dinv.swap(dinv);
        h.A = std::move(A);
        H.lev.push_back(std::move(h));
        A = prune_noise(Cc);                              // coarse operator without residues
    }
    if (H.lev.empty() || A.n > kCoarseDense || !dense_inverse(A, H.ainv)) {
        H = AmgHost();
        return false;
    }
    H.nco = A.n;
    H.nnz_co = (long long)A.col.size();
    return true;
}

// The V-cycle of the device (struct Level) on the host, FP64:
// x = omega D^-1 b, rpre = b - A x, y_{l+1} = cycle(P^T rpre),
// y = omega D^-1 (b + rpre) + U y_{l+1}; the coarsest level y = A^-1 b.
void amg_host_vcycle(const AmgHost& H, size_t l, const double* b, double* y) {
    if (l == H.lev.size()) {
        const int n = H.nco;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += H.ainv[(size_t)i * n + j] * b[j];
            y[i] = s;
        }
        return;
    }
    const AmgHostLevel& V = H.lev[l];
    const int n = V.A.n, nc = V.U.m;
    std::vector<double> x(n), rpre(n), bc(nc), yc(nc);
    for (int i = 0; i < n; ++i) x[i] = V.omega * V.dinv[i] * b[i];
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (long long e = V.A.ptr[i]; e < V.A.ptr[i + 1]; ++e) s += V.A.val[e] * x[V.A.col[e]];
        rpre[i] = b[i] - s;
    }
    for (int I = 0; I < nc; ++I) {                      // P^T (b - A x) = U^T b
        double s = 0.0;
        for (long long e = V.Pt.ptr[I]; e < V.Pt.ptr[I + 1]; ++e) s += V.Pt.val[e] * rpre[V.Pt.col[e]];
        bc[I] = s;
    }
    amg_host_vcycle(H, l + 1, bc.data(), yc.data());
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (long long e = V.U.ptr[i]; e < V.U.ptr[i + 1]; ++e) s += V.U.val[e] * yc[V.U.col[e]];
        y[i] = V.omega * V.dinv[i] * (b[i] + rpre[i]) + s;
    }
}

// The hierarchy of K_phi for the FP32 potential solve: built on the host
// from A, level 0's operator as assembled (before prune_noise; level 0 of
// the hierarchy is its pruned form, which the device holds as P.Kp32),
// uploaded in FP32 (operators SELL-32, P^T CSR).  Leaves P.nlev = 0
// (Jacobi only) when there is none.
int build_hierarchy(mm_ctx* ctx, mm::Problem& P, HostCsr A) {
    int rc;
    P.nlev = 0;
    P.nco = 0;
    P.amg_omega = (float)kAmgOmega;
    ctx->amg_nnz_a.clear();
    ctx->amg_nnz_u.clear();
    ctx->amg_nnz_p.clear();
    const int n0 = P.nphi;
    if (n0 <= kCoarseDense) return MM_OK;
    AmgHost H;
    if (!build_amg_host(std::move(A), H)) return MM_OK;   // Jacobi only
    const int L = (int)H.lev.size();
    for (int l = 0; l < L; ++l) {
        mm::Level& V = P.lev[l];
        const AmgHostLevel& h = H.lev[l];
        V.n = h.U.n;
        V.nc = h.U.m;
        V.omega = (float)h.omega;
        V.wide = (h.Pt.n > 0 && (double)h.Pt.col.size() / h.Pt.n > 160.0) ? 1 : 0;
        V.tab = nullptr;
        if (l == 0) {
            V.sptr = P.k_sptr;
            V.col = P.k_col;
            V.val = P.Kp32;
            V.tab = P.k_tab;
            V.dinv = P.dinvP32;
            V.b = nullptr;
            V.x = nullptr;
            V.y = P.pprec32;
        } else {
            if ((rc = upload_sell(ctx, h.A, &V.sptr, &V.col, &V.val))) return rc;
            std::vector<float> df(h.dinv.begin(), h.dinv.end());
            float* d;
            if ((rc = upload(ctx, &d, df.data(), df.size()))) return rc;
            V.dinv = d;
            if ((rc = dalloc(ctx, &V.b, V.n))) return rc;
            if ((rc = dalloc(ctx, &V.y, V.n))) return rc;
        }
        if ((rc = upload_sell(ctx, h.U, &V.u_sptr, &V.u_col, &V.u_val))) return rc;
        {
            std::vector<float> tv(h.Pt.val.begin(), h.Pt.val.end());
            long long* tp;
            int* tc;
            float* tvd;
            if ((rc = upload(ctx, &tp, h.Pt.ptr.data(), h.Pt.ptr.size()))) return rc;
            if ((rc = upload(ctx, &tc, h.Pt.col.data(), h.Pt.col.size()))) return rc;
            if ((rc = upload(ctx, &tvd, tv.data(), tv.size()))) return rc;
            V.t_ptr = tp;
            V.t_col = tc;
            V.t_val = tvd;
        }
        if (l > 0 && (rc = dalloc(ctx, &V.x, V.n))) return rc;
        if ((rc = dalloc(ctx, &V.rpre, V.n))) return rc;
    }
    if ((rc = dalloc(ctx, &P.amg_x0, n0))) return rc;
    {
        std::vector<float> af(H.ainv.begin(), H.ainv.end());
        float* a;
        if ((rc = upload(ctx, &a, af.data(), af.size()))) return rc;
        P.ainv = a;
    }
    P.nco = H.nco;
    if ((rc = dalloc(ctx, &P.bco, H.nco))) return rc;
    if ((rc = dalloc(ctx, &P.yco, H.nco))) return rc;
    P.nlev = L;
    P.amg_omega = P.lev[0].omega;
    for (const AmgHostLevel& h : H.lev) {
        ctx->amg_nnz_a.push_back((long long)h.A.col.size());
        ctx->amg_nnz_u.push_back((long long)h.U.col.size());
        ctx->amg_nnz_p.push_back((long long)h.Pt.col.size());
    }
    ctx->amg_nnz_a.push_back((long long)H.nco * H.nco);        // the dense inverse
    return MM_OK;
}

// The solver kernel built for `variant` blocks per SM and its grid (as many
// blocks as are co-resident, at most variant per SM).
int select_kernel(mm_ctx* ctx, int variant) {
    ctx->kernel = mm::solver_kernel(variant);
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ctx->kernel, MM_BLOCK, 0) != cudaSuccess || bps < 1) {
        cudaGetLastError();
        return MM_ERR_CUDA;
    }
    ctx->blocks = std::min(bps, variant) * ctx->nsm;
    return MM_OK;
}

// Blocks per SM when the caller left the choice to the library: the phases
// of a potential step are latency-bound, and on GB300 more resident warps
// pay once the mesh is large -- 4 blocks per SM (64 registers) ran the
// 8.7 M-unknown polycrystal 1.26x (multigrid precision form) and 1.30x
// (plain FP64) faster than 2 -- while on the 0.86 M-unknown cube 2 blocks
// per SM (128 registers, fewest spills) were fastest.
constexpr int kAutoLargePhi = 2000000;
int auto_blocks_per_sm(int nphi) { return nphi > kAutoLargePhi ? 4 : 2; }

int launch_solver(mm_ctx* ctx, int mode, const mm::Params& prm) {
    ctx->P.prm = prm;
    ctx->P.mode = mode;
    CK_CUDA(cudaMemsetAsync(ctx->P.bar, 0, 64 * sizeof(unsigned), ctx->stream));
    CK_CUDA(cudaMemsetAsync(ctx->P.err, 0, sizeof(int), ctx->stream));
    void* args[] = {(void*)&ctx->P};
    CK_CUDA(cudaEventRecord(ctx->ev0, ctx->stream));
    CK_CUDA(cudaLaunchCooperativeKernel(ctx->kernel, dim3(ctx->blocks), dim3(MM_BLOCK), args, 0, ctx->stream));
    CK_CUDA(cudaEventRecord(ctx->ev1, ctx->stream));
    CK_CUDA(cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(mm::DevState), cudaMemcpyDeviceToHost,
                            ctx->stream));
    ctx->timed = true;
    return MM_OK;
}

int finish(mm_ctx* ctx) {
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    int e = 0;
    CK_CUDA(cudaMemcpy(&e, ctx->P.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e == mm::ST_TIMEOUT || ctx->h_state->status == mm::ST_TIMEOUT)
        return fail(ctx, MM_ERR_DEVICE_TIMEOUT, "a device barrier wait ran out");
    return MM_OK;
}

void fill_stats(mm_ctx* ctx, mm_stats* out) {
    const mm::DevState& s = *ctx->h_state;
    const double EJ = kMu0 * ctx->Mref * ctx->Mref * 1e-27;
    out->evals = s.evals;
    out->nli = s.nli;
    out->li = s.li;
    out->mi = s.mi;
    out->ls_extra = s.ls_extra;
    out->mr = s.mr;
    out->status = s.status;
    out->pad = 0;
    out->F = s.F * EJ;
    for (int k = 0; k < 4; ++k) out->terms[k] = s.terms[k] * EJ;
    out->F_internal = s.F;
    for (int k = 0; k < 3; ++k) out->M[k] = s.M[k];
    out->li2 = s.li2;
    out->li2_first = s.li2_first;
    out->restarts = s.restarts;
    out->steepest = s.steepest;
}

int status_code(int st) {
    switch (st) {
        case mm::ST_OK: return MM_OK;
        case mm::ST_NOT_CONVERGED: return MM_NOT_CONVERGED;
        case mm::ST_STALLED: return MM_STALLED;
        case mm::ST_NONFINITE: return MM_ERR_NONFINITE;
        case mm::ST_TIMEOUT: return MM_ERR_DEVICE_TIMEOUT;
        default: return MM_ERR_STATE;
    }
}

int need_mesh(mm_ctx* ctx) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->has_mesh) return fail(ctx, MM_ERR_STATE, "no mesh uploaded");
    CK_CUDA(cudaSetDevice(ctx->device));
    return MM_OK;
}

int set_m_from_stage(mm_ctx* ctx) {
    CK_CUDA(cudaStreamSynchronize(ctx->stream));   // h_state->cur is current after this
    CK_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    k_set_m<<<nblk(ctx->nm), 256, 0, ctx->stream>>>(ctx->nm, ctx->d_mag_nodes, ctx->d_stage,
                                                     ctx->P.X[ctx->h_state->cur], ctx->d_flag);
    CK_CUDA(cudaGetLastError());
    int bad = 0;
    CK_CUDA(cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->has_eval = false;
    if (bad) return fail(ctx, MM_ERR_NONFINITE, "magnetisation has a zero or non-finite vector");
    return MM_OK;
}

int eval_current(mm_ctx* ctx, const mm_params* p) {
    int rc = check_params(ctx, p);
    if (rc) return rc;
    rc = launch_solver(ctx, mm::MODE_EVAL, to_params(p));
    if (rc) return rc;
    rc = finish(ctx);
    if (rc) return rc;
    ctx->has_eval = true;
    if (!std::isfinite(ctx->h_state->F)) return fail(ctx, MM_ERR_NONFINITE, "non-finite energy");
    return MM_OK;
}

int maybe_set_m(mm_ctx* ctx, const double* m) {
    if (!m) return MM_OK;
    CK_CUDA(cudaMemcpy(ctx->d_stage, m, (size_t)ctx->n_nodes * 3 * sizeof(double), cudaMemcpyHostToDevice));
    return set_m_from_stage(ctx);
}

int copy_out3(mm_ctx* ctx, const double* dev_soa, double* host) {
    CK_CUDA(cudaMemsetAsync(ctx->d_stage, 0, (size_t)ctx->n_nodes * 3 * sizeof(double), ctx->stream));
    k_scatter3<<<nblk(ctx->nm), 256, 0, ctx->stream>>>(ctx->nm, ctx->d_mag_nodes, dev_soa, ctx->d_stage);
    CK_CUDA(cudaGetLastError());
    CK_CUDA(cudaMemcpyAsync(host, ctx->d_stage, (size_t)ctx->n_nodes * 3 * sizeof(double),
                            cudaMemcpyDeviceToHost, ctx->stream));
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

}  // namespace

namespace mm {

const void* solver_kernel_2();
const void* solver_kernel_3();
const void* solver_kernel_4();
const void* solver_batch_kernel_2();
const void* solver_batch_kernel_3();
const void* solver_batch_kernel_4();

const void* solver_kernel(int min_blocks) {
    switch (min_blocks) {
        case 2: return solver_kernel_2();
        case 4: return solver_kernel_4();
        default: return solver_kernel_3();
    }
}

const void* solver_batch_kernel(int min_blocks) {
    return min_blocks == 4 ? solver_batch_kernel_4() : min_blocks == 2 ? solver_batch_kernel_2() : solver_batch_kernel_3();
}

int ctx_view(mm_ctx* ctx, CtxView* out) {
    if (!ctx || !out) return MM_ERR_ARG;
    out->P = &ctx->P;
    out->stream = (void*)ctx->stream;
    out->device = ctx->device;
    out->blocks = ctx->blocks;
    out->n_nodes = ctx->n_nodes;
    out->nm = ctx->nm;
    out->nphi = ctx->nphi;
    out->Mref = ctx->Mref;
    for (int k = 0; k < 3; ++k) out->field_T[k] = ctx->field_T[k];
    out->mag_nodes = ctx->d_mag_nodes;
    out->node_of_phi = ctx->d_node_of_phi;
    out->ident = ctx->d_ident;
    out->has_mesh = ctx->has_mesh;
    out->kernel = ctx->kernel;
    out->d_state = ctx->d_state;
    out->nnz_mag = ctx->nnzm_true;
    out->nnz_phi = ctx->nnzp_true;
    return MM_OK;
}

int ctx_fail(mm_ctx* ctx, int code, const char* msg) { return fail(ctx, code, "%s", msg); }

int ctx_refresh_state(mm_ctx* ctx) {
    if (!ctx || !ctx->has_mesh) return MM_ERR_STATE;
    CK_CUDA(cudaSetDevice(ctx->device));
    CK_CUDA(cudaMemcpy(ctx->h_state, ctx->d_state, sizeof(mm::DevState), cudaMemcpyDeviceToHost));
    ctx->has_eval = true;
    return MM_OK;
}

}  // namespace mm

extern "C" {

void mm_default_params(mm_params* p) {
    if (!p) return;
    p->tau_F = 1e-10;
    p->jmax = 4;
    p->max_iter = 10000;
    p->theta_max = 0.1;
    p->c1 = 1e-4;
    p->max_backtrack = 10;
    p->keep_last_term = 0;
    p->poisson_tol = 1e-10;
    p->poisson_max_iter = 20000;
    p->precision = 0;
    p->inner_tol = 0.1;
    p->max_refine = 64;
    p->amg = 0;
    p->beta_rule = 0;
    p->poisson_sched = 0;
    p->poisson_tol_max = 1e-6;
}

int mm_create(mm_ctx** out, const mm_options* opt) {
    if (!out) return MM_ERR_ARG;
    *out = nullptr;
    mm_ctx* ctx = new mm_ctx();
    ctx->device = opt ? opt->device : 0;
    ctx->blocks_per_sm_req = opt ? opt->blocks_per_sm : 0;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        delete ctx;
        return MM_ERR_CUDA;
    }
    if (ctx->device < 0 || ctx->device >= ndev) {
        delete ctx;
        return MM_ERR_ARG;
    }
    auto bail = [&](int code) {
        delete ctx;
        return code;
    };
    if (cudaSetDevice(ctx->device) != cudaSuccess) return bail(MM_ERR_CUDA);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (!coop) return bail(MM_ERR_CUDA);
    cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    // blocks_per_sm selects the kernel instantiation (register budget) and
    // the grid: 2, 3 or 4 blocks per SM; 0 = chosen by mm_upload_mesh from
    // the mesh size (select_kernel), 2 until then.
    const int variant = (ctx->blocks_per_sm_req >= 2 && ctx->blocks_per_sm_req <= 4) ? ctx->blocks_per_sm_req : 2;
    if (select_kernel(ctx, variant) != MM_OK) return bail(MM_ERR_CUDA);
    if (opt && opt->stream) {
        ctx->stream = (cudaStream_t)opt->stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(MM_ERR_CUDA);
        ctx->own_stream = true;
    }
    if (cudaMalloc(&ctx->d_state, sizeof(mm::DevState)) != cudaSuccess) return bail(MM_ERR_OOM);
    if (cudaMallocHost(&ctx->h_state, sizeof(mm::DevState)) != cudaSuccess) return bail(MM_ERR_OOM);
    if (cudaMalloc(&ctx->d_flag, sizeof(int)) != cudaSuccess) return bail(MM_ERR_OOM);
    std::memset(ctx->h_state, 0, sizeof(mm::DevState));
    cudaMemset(ctx->d_state, 0, sizeof(mm::DevState));
    cudaEventCreate(&ctx->ev0);
    cudaEventCreate(&ctx->ev1);
    *out = ctx;
    return MM_OK;
}

void mm_destroy(mm_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_mesh(ctx);
    if (ctx->d_state) cudaFree(ctx->d_state);
    if (ctx->h_state) cudaFreeHost(ctx->h_state);
    if (ctx->d_flag) cudaFree(ctx->d_flag);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* mm_last_error(const mm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void* mm_stream(const mm_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

int mm_upload_mesh(mm_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_tets, const int32_t* tets,
                   const int32_t* region, int32_t n_regions, const mm_material* materials) {
    if (!ctx) return MM_ERR_ARG;
    if (!xyz || !tets || !region || !materials) return fail(ctx, MM_ERR_ARG, "null array");
    if (n_nodes < 4 || n_tets < 1 || n_regions < 1) return fail(ctx, MM_ERR_ARG, "empty mesh");
    if (n_nodes >= (1ll << 31) - 64 || n_tets >= (1ll << 31) / 4)
        return fail(ctx, MM_ERR_ARG, "mesh too large for 32-bit indices");
    CK_CUDA(cudaSetDevice(ctx->device));
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    free_mesh(ctx);
    const long long N = n_nodes, T = n_tets;
    // ---- validation
    double Mref = 0.0;
    std::vector<double> mat(6 * (size_t)n_regions);
    for (int r = 0; r < n_regions; ++r) {
        const mm_material& m = materials[r];
        const double an = std::sqrt(m.axis[0] * m.axis[0] + m.axis[1] * m.axis[1] + m.axis[2] * m.axis[2]);
        if (!std::isfinite(m.Ms) || !std::isfinite(m.A) || !std::isfinite(m.K1) || m.Ms < 0 || m.A < 0)
            return fail(ctx, MM_ERR_ARG, "material %d: Ms, A must be finite and >= 0, K1 finite", r);
        if (m.Ms > 0 && !(an > 0 && std::isfinite(an)))
            return fail(ctx, MM_ERR_ARG, "material %d: easy axis must be non-zero", r);
        mat[6 * r] = m.Ms;
        mat[6 * r + 1] = m.A;
        mat[6 * r + 2] = m.K1;
        mat[6 * r + 3] = an > 0 ? m.axis[0] : 0.0;
        mat[6 * r + 4] = an > 0 ? m.axis[1] : 0.0;
        mat[6 * r + 5] = an > 0 ? m.axis[2] : 1.0;
        Mref = std::max(Mref, m.Ms);
    }
    if (!(Mref > 0)) return fail(ctx, MM_ERR_ARG, "no magnetic material (all Ms = 0)");
    for (long long i = 0; i < 3 * N; ++i)
        if (!std::isfinite(xyz[i])) return fail(ctx, MM_ERR_MESH, "non-finite coordinate");
    std::vector<long long> cnt(N + 1, 0);
    for (long long e = 0; e < T; ++e) {
        if (region[e] < 0 || region[e] >= n_regions) return fail(ctx, MM_ERR_MESH, "tet %lld: bad region", e);
        for (int v = 0; v < 4; ++v) {
            const int n = tets[4 * e + v];
            if (n < 0 || n >= N) return fail(ctx, MM_ERR_MESH, "tet %lld: node index out of range", e);
            for (int u = 0; u < v; ++u)
                if (tets[4 * e + u] == n) return fail(ctx, MM_ERR_MESH, "tet %lld: repeated node", e);
            cnt[n + 1]++;
        }
    }
    // node -> incident tets, ascending tet order
    for (long long n = 0; n < N; ++n) cnt[n + 1] += cnt[n];
    std::vector<long long> nt_ptr = cnt;
    std::vector<int> nt_idx(4 * T);
    {
        std::vector<long long> fillp(nt_ptr.begin(), nt_ptr.end() - 1);
        for (long long e = 0; e < T; ++e)
            for (int v = 0; v < 4; ++v) nt_idx[fillp[tets[4 * e + v]]++] = (int)e;
    }
    // magnetic nodes
    std::vector<int> mag_of(N, -1), mag_nodes;
    {
        std::vector<char> ismag(N, 0);
        for (long long e = 0; e < T; ++e)
            if (mat[6 * region[e]] > 0)
                for (int v = 0; v < 4; ++v) ismag[tets[4 * e + v]] = 1;
        for (long long n = 0; n < N; ++n)
            if (ismag[n]) {
                mag_of[n] = (int)mag_nodes.size();
                mag_nodes.push_back((int)n);
            }
    }
    const int nm = (int)mag_nodes.size();
    // outer surface: faces that belong to exactly one tet
    std::vector<char> dirichlet(N, 0);
    {
        std::vector<std::array<int, 3>> faces;
        faces.reserve(4 * T);
        for (long long e = 0; e < T; ++e) {
            const int* t = tets + 4 * e;
            for (int skip = 0; skip < 4; ++skip) {
                std::array<int, 3> f;
                int q = 0;
                for (int v = 0; v < 4; ++v)
                    if (v != skip) f[q++] = t[v];
                std::sort(f.begin(), f.end());
                faces.push_back(f);
            }
        }
        std::sort(faces.begin(), faces.end());
        size_t i = 0;
        while (i < faces.size()) {
            size_t j = i + 1;
            while (j < faces.size() && faces[j] == faces[i]) ++j;
            if (j - i == 1)
                for (int v = 0; v < 3; ++v) dirichlet[faces[i][v]] = 1;
            else if (j - i > 2)
                return fail(ctx, MM_ERR_MESH, "a face is shared by more than two tets");
            i = j;
        }
    }
    // potential numbering: magnetic nodes first (identity rows where on the
    // outer surface), then free air nodes in ascending node id
    std::vector<int> phi_of(N, -1), node_of_phi;
    std::vector<unsigned char> ident;
    for (int i = 0; i < nm; ++i) {
        phi_of[mag_nodes[i]] = i;
        node_of_phi.push_back(mag_nodes[i]);
        ident.push_back(dirichlet[mag_nodes[i]] ? 1 : 0);
    }
    for (long long n = 0; n < N; ++n)
        if (mag_of[n] < 0 && !dirichlet[n]) {
            phi_of[n] = (int)node_of_phi.size();
            node_of_phi.push_back((int)n);
            ident.push_back(0);
        }
    const int nphi = (int)node_of_phi.size();
    // adjacency lists
    std::vector<std::vector<int>> prow(nphi), mrow(nm);
    for (int p = 0; p < nphi; ++p) {
        auto& r = prow[p];
        if (ident[p]) {
            r.push_back(p);
            continue;
        }
        const int n = node_of_phi[p];
        for (long long q = nt_ptr[n]; q < nt_ptr[n + 1]; ++q) {
            const int e = nt_idx[q];
            for (int v = 0; v < 4; ++v) {
                const int pc = phi_of[tets[4ll * e + v]];
                if (pc >= 0 && !ident[pc]) r.push_back(pc);
            }
        }
        r.push_back(p);
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
    }
    for (int i = 0; i < nm; ++i) {
        auto& r = mrow[i];
        const int n = mag_nodes[i];
        for (long long q = nt_ptr[n]; q < nt_ptr[n + 1]; ++q) {
            const int e = nt_idx[q];
            if (!(mat[6 * region[e]] > 0)) continue;
            for (int v = 0; v < 4; ++v) r.push_back(mag_of[tets[4ll * e + v]]);
        }
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
    }
    std::vector<long long> m_sptr, p_sptr;
    std::vector<int> m_col, p_col;
    long long nnzm_true = 0, nnzp_true = 0;
    build_sell(mrow, m_sptr, m_col, nnzm_true);
    build_sell(prow, p_sptr, p_col, nnzp_true);
    mrow.clear();
    prow.clear();
    const long long nnzm = m_sptr.back(), nnzp_asm = p_sptr.back();

    // ---- device upload and assembly
    int rc;
    double *d_xyz, *d_mat, *d_vol, *d_grad;
    int *d_tets, *d_region, *d_nt_idx, *d_mag_of, *d_phi_of;
    long long* d_nt_ptr;
    mm::Problem& P = ctx->P;
    P.nm = nm;
    P.nphi = nphi;
    P.nnzm = nnzm;
    // the mesh arrays only live for the assembly: allocate them last-freed
    std::vector<void*> tmp_start(ctx->allocs);
    if ((rc = upload(ctx, &d_xyz, xyz, 3 * N))) return rc;
    if ((rc = upload(ctx, &d_tets, (const int*)tets, 4 * T))) return rc;
    if ((rc = upload(ctx, &d_region, (const int*)region, T))) return rc;
    if ((rc = upload(ctx, &d_mat, mat.data(), mat.size()))) return rc;
    if ((rc = upload(ctx, &d_nt_ptr, nt_ptr.data(), nt_ptr.size()))) return rc;
    if ((rc = upload(ctx, &d_nt_idx, nt_idx.data(), nt_idx.size()))) return rc;
    if ((rc = upload(ctx, &d_mag_of, mag_of.data(), mag_of.size()))) return rc;
    if ((rc = upload(ctx, &d_phi_of, phi_of.data(), phi_of.size()))) return rc;
    if ((rc = dalloc(ctx, &d_vol, T))) return rc;
    if ((rc = dalloc(ctx, &d_grad, 12 * T))) return rc;
    const size_t n_tmp = ctx->allocs.size() - tmp_start.size();
    // persistent arrays
    long long *d_msp, *d_psp;
    int *d_mcol, *d_pcol;
    double *KA, *G, *B, *CK, *w, *dinvA, *Kp, *dinvP;
    if ((rc = upload(ctx, &ctx->d_mag_nodes, mag_nodes.data(), mag_nodes.size()))) return rc;
    if ((rc = upload(ctx, &ctx->d_node_of_phi, node_of_phi.data(), node_of_phi.size()))) return rc;
    if ((rc = upload(ctx, &ctx->d_ident, ident.data(), ident.size()))) return rc;
    if ((rc = upload(ctx, &d_msp, m_sptr.data(), m_sptr.size()))) return rc;
    if ((rc = upload(ctx, &d_mcol, m_col.data(), m_col.size()))) return rc;
    if ((rc = upload(ctx, &d_psp, p_sptr.data(), p_sptr.size()))) return rc;
    if ((rc = upload(ctx, &d_pcol, p_col.data(), p_col.size()))) return rc;
    if ((rc = dalloc(ctx, &KA, nnzm))) return rc;
    if ((rc = dalloc(ctx, &G, 3 * nnzm))) return rc;
    if ((rc = dalloc(ctx, &B, 3 * nnzm))) return rc;
    if ((rc = dalloc(ctx, &CK, 6 * (size_t)nm))) return rc;
    if ((rc = dalloc(ctx, &w, nm))) return rc;
    if ((rc = dalloc(ctx, &dinvA, nm))) return rc;
    if ((rc = dalloc(ctx, &Kp, nnzp_asm))) return rc;
    if ((rc = dalloc(ctx, &dinvP, nphi))) return rc;
    CK_CUDA(cudaMemset(ctx->d_flag, 0, sizeof(int)));
    mm::k_tet_geometry<<<nblk(T), 256, 0, ctx->stream>>>(T, d_xyz, d_tets, d_vol, d_grad, ctx->d_flag);
    CK_CUDA(cudaGetLastError());
    mm::AssembleArgs A;
    A.nm = nm;
    A.nphi = nphi;
    A.Mref = Mref;
    A.tets = d_tets;
    A.region = d_region;
    A.materials = d_mat;
    A.vol = d_vol;
    A.grad = d_grad;
    A.nt_ptr = d_nt_ptr;
    A.nt_idx = d_nt_idx;
    A.mag_of = d_mag_of;
    A.phi_of = d_phi_of;
    A.mag_nodes = ctx->d_mag_nodes;
    A.node_of_phi = ctx->d_node_of_phi;
    A.phi_ident = ctx->d_ident;
    A.m_sptr = d_msp;
    A.m_col = d_mcol;
    A.nnzm = nnzm;
    A.KA = KA;
    A.G = G;
    A.B = B;
    A.CK = CK;
    A.w = w;
    A.dinvA = dinvA;
    A.p_sptr = d_psp;
    A.p_col = d_pcol;
    A.Kp = Kp;
    A.dinvP = dinvP;
    A.bad = ctx->d_flag;
    mm::k_assemble_phi<<<nblk(nphi), 256, 0, ctx->stream>>>(A);
    CK_CUDA(cudaGetLastError());
    mm::k_assemble_mag<<<nblk(nm), 256, 0, ctx->stream>>>(A);
    CK_CUDA(cudaGetLastError());
    int bad = 0;
    CK_CUDA(cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    // free the assembly-only arrays
    for (size_t k = 0; k < n_tmp; ++k) cudaFree(ctx->allocs[tmp_start.size() + k]);
    ctx->allocs.erase(ctx->allocs.begin() + tmp_start.size(), ctx->allocs.begin() + tmp_start.size() + n_tmp);
    if (bad == 1) {
        free_mesh(ctx);
        return fail(ctx, MM_ERR_MESH, "degenerate tetrahedron (zero volume)");
    }
    if (bad) {
        free_mesh(ctx);
        return fail(ctx, MM_ERR_MESH, "assembly failed (code %d)", bad);
    }
    // ---- the potential stiffness without its rounding residues
    // (prune_noise): download, compact, upload again in SELL-32
    HostCsr Kfull;
    {
        std::vector<double> kp(nnzp_asm);
        CK_CUDA(cudaMemcpy(kp.data(), Kp, nnzp_asm * sizeof(double), cudaMemcpyDeviceToHost));
        Kfull.n = Kfull.m = nphi;
        Kfull.ptr.assign(nphi + 1, 0);
        Kfull.col.reserve(nnzp_true);
        Kfull.val.reserve(nnzp_true);
        for (int r = 0; r < nphi; ++r) {
            const long long sl = r / 32, w = (p_sptr[sl + 1] - p_sptr[sl]) / 32;
            for (long long k = 0; k < w; ++k) {
                const long long e = p_sptr[sl] + 32 * k + (r % 32);
                if (p_col[e] == r && kp[e] == 0.0) continue;   // SELL padding
                Kfull.col.push_back(p_col[e]);
                Kfull.val.push_back(kp[e]);
            }
            Kfull.ptr[r + 1] = (long long)Kfull.col.size();
        }
    }
    K32Layout K32;
    {
        const HostCsr Kpr = prune_noise(Kfull);
        K32 = k32_layout(Kpr);
        std::vector<double> v;
        csr_to_sell(Kpr, p_sptr, p_col, v);
        dfree(ctx, d_psp);
        dfree(ctx, d_pcol);
        dfree(ctx, Kp);
        if ((rc = upload(ctx, &d_psp, p_sptr.data(), p_sptr.size()))) return rc;
        if ((rc = upload(ctx, &d_pcol, p_col.data(), p_col.size()))) return rc;
        if ((rc = upload(ctx, &Kp, v.data(), v.size()))) return rc;
        nnzp_true = (long long)Kpr.col.size();
    }
    const long long nnzp = p_sptr.back();
    P.m_sptr = d_msp;
    P.m_col = d_mcol;
    P.KA = KA;
    P.G = G;
    P.B = B;
    P.CK = CK;
    P.w = w;
    P.dinvA = dinvA;
    P.p_sptr = d_psp;
    P.p_col = d_pcol;
    P.Kp = Kp;
    P.dinvP = dinvP;
    // solver vectors
    const size_t v3 = 3 * (size_t)nm;
    for (int s = 0; s < MM_NSLOT; ++s) {
        if ((rc = dalloc(ctx, &P.X[s], v3))) return rc;
        if ((rc = dalloc(ctx, &P.GR[s], v3))) return rc;
        if ((rc = dalloc(ctx, &P.GP[s], v3))) return rc;
        if ((rc = dalloc(ctx, &P.LAM[s], nm))) return rc;
    }
    if ((rc = dalloc(ctx, &P.unorm, nm))) return rc;
    if ((rc = dalloc(ctx, &P.d, v3))) return rc;
    if ((rc = dalloc(ctx, &P.isol, v3))) return rc;
    if ((rc = dalloc(ctx, &P.ires, v3))) return rc;
    if ((rc = dalloc(ctx, &P.iprec, v3))) return rc;
    if ((rc = dalloc(ctx, &P.idir[0], v3))) return rc;
    if ((rc = dalloc(ctx, &P.idir[1], v3))) return rc;
    if ((rc = dalloc(ctx, &P.ihd, v3))) return rc;
    {
        // FP32 copies for the precision form's preconditioner apply
        float *ka32, *ck32, *da32;
        if ((rc = dalloc(ctx, &ka32, nnzm))) return rc;
        if ((rc = dalloc(ctx, &ck32, 6 * (size_t)nm))) return rc;
        if ((rc = dalloc(ctx, &da32, nm))) return rc;
        k_to_f32<<<nblk(nnzm), 256, 0, ctx->stream>>>(nnzm, KA, ka32);
        k_to_f32<<<nblk(6 * (long long)nm), 256, 0, ctx->stream>>>(6 * (long long)nm, CK, ck32);
        k_to_f32<<<nblk(nm), 256, 0, ctx->stream>>>(nm, dinvA, da32);
        CK_CUDA(cudaGetLastError());
        P.KA32 = ka32;
        P.CK32 = ck32;
        P.dinvA32 = da32;
        if ((rc = dalloc(ctx, &P.ires32, v3))) return rc;
        if ((rc = dalloc(ctx, &P.iprec32, v3))) return rc;
        if ((rc = dalloc(ctx, &P.idir32, v3))) return rc;
        if ((rc = dalloc(ctx, &P.ihd32, v3))) return rc;
    }
    if ((rc = dalloc(ctx, &P.phi, nphi))) return rc;
    for (int s = 0; s < MM_NSLOT; ++s)
        if ((rc = dalloc(ctx, &P.PHI[s], nphi))) return rc;
    if ((rc = dalloc(ctx, &P.rhs, nm))) return rc;
    if ((rc = dalloc(ctx, &P.pres, nphi))) return rc;
    if ((rc = dalloc(ctx, &P.pprec, nphi))) return rc;
    if ((rc = dalloc(ctx, &P.pdir[0], nphi))) return rc;
    if ((rc = dalloc(ctx, &P.pdir[1], nphi))) return rc;
    if ((rc = dalloc(ctx, &P.pq, nphi))) return rc;
    {
        float *k32, *d32;
        long long* ksp;
        int *kcol, *ktab;
        if ((rc = upload(ctx, &ksp, K32.sptr.data(), K32.sptr.size()))) return rc;
        if ((rc = upload(ctx, &kcol, K32.col.data(), K32.col.size()))) return rc;
        if ((rc = upload(ctx, &ktab, K32.tab.data(), K32.tab.size()))) return rc;
        if ((rc = upload(ctx, &k32, K32.val.data(), K32.val.size()))) return rc;
        if ((rc = dalloc(ctx, &d32, nphi))) return rc;
        k_to_f32<<<nblk(nphi), 256, 0, ctx->stream>>>(nphi, dinvP, d32);
        CK_CUDA(cudaGetLastError());
        P.k_sptr = ksp;
        P.k_col = kcol;
        P.k_tab = ktab;
        P.Kp32 = k32;
        P.dinvP32 = d32;
        ctx->k32_slices = (long long)K32.sptr.size() - 1;
        ctx->k32_table_slices = K32.table_slices;
        ctx->k32_bytes = K32.bytes;
        K32 = K32Layout{};
        if ((rc = dalloc(ctx, &P.pres32, nphi))) return rc;
        if ((rc = dalloc(ctx, &P.pprec32, nphi))) return rc;
        if ((rc = dalloc(ctx, &P.pdir32, nphi))) return rc;
        if ((rc = dalloc(ctx, &P.pq32, nphi))) return rc;
        if ((rc = dalloc(ctx, &P.pdelta32, nphi))) return rc;
        for (float* f : {P.pres32, P.pprec32, P.pdir32, P.pq32, P.pdelta32})
            CK_CUDA(cudaMemsetAsync(f, 0, nphi * sizeof(float), ctx->stream));
    }
    // aggregation multigrid hierarchy of K_phi for the FP32 potential solve
    if ((rc = build_hierarchy(ctx, P, std::move(Kfull)))) return rc;
    if (ctx->blocks_per_sm_req < 2 || ctx->blocks_per_sm_req > 4) {
        if (select_kernel(ctx, auto_blocks_per_sm(nphi)) != MM_OK) return fail(ctx, MM_ERR_CUDA, "no solver grid");
    }
    if ((rc = dalloc(ctx, &P.partials, 2 * (size_t)MM_MAXRED * ctx->blocks))) return rc;
    if ((rc = dalloc(ctx, &P.bar, 64))) return rc;
    if ((rc = dalloc(ctx, &P.err, 1))) return rc;
    if ((rc = dalloc(ctx, &ctx->d_stage, 3 * (size_t)N))) return rc;
    P.state = ctx->d_state;
    // zero every solver vector once (directions are read with coefficient
    // 0 only behind explicit branches, but keep them finite regardless)
    auto z = [&](double* p, size_t n) { return cudaMemsetAsync(p, 0, n * sizeof(double), ctx->stream); };
    for (int s = 0; s < MM_NSLOT; ++s) {
        CK_CUDA(z(P.X[s], v3));
        CK_CUDA(z(P.GR[s], v3));
        CK_CUDA(z(P.GP[s], v3));
        CK_CUDA(z(P.LAM[s], nm));
    }
    CK_CUDA(z(P.unorm, nm));
    CK_CUDA(z(P.d, v3));
    CK_CUDA(z(P.isol, v3));
    CK_CUDA(z(P.ires, v3));
    CK_CUDA(z(P.iprec, v3));
    CK_CUDA(z(P.idir[0], v3));
    CK_CUDA(z(P.idir[1], v3));
    CK_CUDA(z(P.ihd, v3));
    for (float* f : {P.ires32, P.iprec32, P.idir32, P.ihd32})
        CK_CUDA(cudaMemsetAsync(f, 0, v3 * sizeof(float), ctx->stream));
    CK_CUDA(z(P.phi, nphi));
    for (int s = 0; s < MM_NSLOT; ++s) CK_CUDA(z(P.PHI[s], nphi));
    CK_CUDA(z(P.rhs, nm));
    CK_CUDA(z(P.pres, nphi));
    CK_CUDA(z(P.pprec, nphi));
    CK_CUDA(z(P.pdir[0], nphi));
    CK_CUDA(z(P.pdir[1], nphi));
    CK_CUDA(z(P.pq, nphi));
    ctx->n_nodes = N;
    ctx->nm = nm;
    ctx->nphi = nphi;
    ctx->nnzm = nnzm;
    ctx->nnzp = nnzp;
    ctx->nnzm_true = nnzm_true;
    ctx->nnzp_true = nnzp_true;
    ctx->Mref = Mref;
    ctx->has_mesh = true;
    // initial state: m = +z, zero field, slot 0
    std::memset(ctx->h_state, 0, sizeof(mm::DevState));
    CK_CUDA(cudaMemsetAsync(ctx->d_state, 0, sizeof(mm::DevState), ctx->stream));
    k_set_cur<<<1, 1, 0, ctx->stream>>>(ctx->d_state, 0);
    k_set_field<<<1, 1, 0, ctx->stream>>>(ctx->d_state, 0.0, 0.0, 0.0);
    ctx->field_T[0] = ctx->field_T[1] = ctx->field_T[2] = 0.0;
    std::vector<double> mz(3 * (size_t)N, 0.0);
    for (long long n = 0; n < N; ++n) mz[3 * n + 2] = 1.0;
    CK_CUDA(cudaMemcpy(ctx->d_stage, mz.data(), mz.size() * sizeof(double), cudaMemcpyHostToDevice));
    return set_m_from_stage(ctx);
}

int mm_coercive_field(int64_t n, const double* fields, const double* M, double* hc_out, int32_t* found) {
    if (n < 2 || !fields || !M || !hc_out || !found) return MM_ERR_ARG;
    for (int64_t k = 0; k < 3 * n; ++k)
        if (!std::isfinite(fields[k]) || !std::isfinite(M[k])) return MM_ERR_ARG;
    const double* f0 = fields;
    const double* f1 = fields + 3 * (n - 1);
    double u[3] = {f1[0] - f0[0], f1[1] - f0[1], f1[2] - f0[2]};
    double nu = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (nu == 0.0) {
        for (int c = 0; c < 3; ++c) u[c] = f1[c];
        nu = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    }
    if (!(nu > 0.0)) return MM_ERR_ARG;
    for (int c = 0; c < 3; ++c) u[c] /= nu;
    auto along = [&](const double* v, int64_t k) {
        return v[3 * k] * u[0] + v[3 * k + 1] * u[1] + v[3 * k + 2] * u[2];
    };
    *found = 0;
    for (int64_t k = 1; k < n; ++k) {
        const double ma = along(M, k - 1), mb = along(M, k);
        const double ha = along(fields, k - 1), hb = along(fields, k);
        if (ma == 0.0) {
            *hc_out = std::fabs(ha);
            *found = 1;
            return MM_OK;
        }
        if (ma * mb < 0.0) {
            const double t = ma / (ma - mb);
            *hc_out = std::fabs(ha + t * (hb - ha));
            *found = 1;
            return MM_OK;
        }
    }
    return MM_OK;
}

int mm_sizes(const mm_ctx* ctx, int64_t* n_mag, int64_t* n_phi, int64_t* nnz_mag, int64_t* nnz_phi) {
    if (!ctx || !ctx->has_mesh) return MM_ERR_STATE;
    if (n_mag) *n_mag = ctx->nm;
    if (n_phi) *n_phi = ctx->nphi;
    if (nnz_mag) *nnz_mag = ctx->nnzm_true;
    if (nnz_phi) *nnz_phi = ctx->nnzp_true;
    return MM_OK;
}

int mm_amg_info(const mm_ctx* ctx, int32_t* n_levels, int64_t* rows, int64_t* nnz_a, int64_t* nnz_u,
                int64_t* nnz_p, int32_t max_entries) {
    if (!ctx || !ctx->has_mesh) return MM_ERR_STATE;
    const mm::Problem& P = ctx->P;
    if (n_levels) *n_levels = P.nlev;
    if (P.nlev == 0) return MM_OK;
    for (int l = 0; l <= P.nlev && l < max_entries; ++l) {
        if (rows) rows[l] = (l < P.nlev) ? P.lev[l].n : P.nco;
        if (nnz_a) nnz_a[l] = ctx->amg_nnz_a[l];
        if (nnz_u && l < P.nlev) nnz_u[l] = ctx->amg_nnz_u[l];
        if (nnz_p && l < P.nlev) nnz_p[l] = ctx->amg_nnz_p[l];
    }
    return MM_OK;
}

int mm_k32_layout_info(const mm_ctx* ctx, int64_t* slices, int64_t* table_slices, int64_t* matrix_bytes) {
    if (!ctx || !ctx->has_mesh) return MM_ERR_STATE;
    if (slices) *slices = ctx->k32_slices;
    if (table_slices) *table_slices = ctx->k32_table_slices;
    if (matrix_bytes) *matrix_bytes = ctx->k32_bytes;
    return MM_OK;
}

int mm_k32_host_apply(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val, const float* x,
                      float* y, int64_t* table_slices, int64_t* matrix_bytes) {
    if (n < 1 || n > INT32_MAX || !row_ptr || !col || !val || !x || !y) return MM_ERR_ARG;
    if (row_ptr[0] != 0) return MM_ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return MM_ERR_ARG;
    HostCsr A;
    A.n = A.m = (int)n;
    A.ptr.assign(row_ptr, row_ptr + n + 1);
    const long long nnz = A.ptr[n];
    A.col.resize(nnz);
    A.val.resize(nnz);
    for (long long e = 0; e < nnz; ++e) {
        if (col[e] < 0 || col[e] >= n) return MM_ERR_ARG;
        A.col[e] = col[e];
        A.val[e] = val[e];
    }
    const K32Layout L = k32_layout(prune_noise(A));
    if (table_slices) *table_slices = L.table_slices;
    if (matrix_bytes) *matrix_bytes = L.bytes;
    // the device's entry order: entry k of row r at sptr[s] + 32 k + (r % 32)
    for (long long r = 0; r < n; ++r) {
        const long long s = r / 32, w = (L.sptr[s + 1] - L.sptr[s]) / 32;
        const bool tab = L.tab[s * 8] != MM_NO_TAB;
        float acc = 0.0f;
        for (long long k = 0; k < w; ++k) {
            const long long e = L.sptr[s] + 32 * k + (r % 32);
            const long long c = tab ? r + L.tab[s * 8 + k] : L.col[e];
            acc += L.val[e] * x[c];
        }
        y[r] = acc;
    }
    return MM_OK;
}

int mm_amg_host_apply(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val, int32_t n_vec,
                      const double* r, double* z, int32_t* n_levels, int64_t* rows, int32_t max_rows) {
    if (n < 1 || n > INT32_MAX || !row_ptr || !col || !val || n_vec < 0 || (n_vec > 0 && (!r || !z)))
        return MM_ERR_ARG;
    if (row_ptr[0] != 0) return MM_ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return MM_ERR_ARG;
    HostCsr A;
    A.n = A.m = (int)n;
    A.ptr.assign(row_ptr, row_ptr + n + 1);
    const long long nnz = A.ptr[n];
    A.col.resize(nnz);
    A.val.resize(nnz);
    for (long long e = 0; e < nnz; ++e) {
        if (col[e] < 0 || col[e] >= n) return MM_ERR_ARG;
        A.col[e] = col[e];
        A.val[e] = val[e];
    }
    AmgHost H;
    const bool ok = build_amg_host(std::move(A), H);
    const int L = ok ? (int)H.lev.size() : 0;
    if (n_levels) *n_levels = L;
    if (!ok) return MM_OK;
    for (int l = 0; l <= L && rows && l < max_rows; ++l) rows[l] = (l < L) ? H.lev[l].A.n : H.nco;
    for (int32_t v = 0; v < n_vec; ++v) amg_host_vcycle(H, 0, r + (size_t)v * n, z + (size_t)v * n);
    return MM_OK;
}

int mm_set_tiles(mm_ctx* ctx, int32_t rows_per_thread, int32_t restrict_lanes) {
    if (!ctx) return MM_ERR_ARG;
    if (rows_per_thread < 0 || rows_per_thread > 2) return fail(ctx, MM_ERR_ARG, "rows_per_thread must be 0, 1 or 2");
    if (restrict_lanes != 0 && restrict_lanes != 4 && restrict_lanes != 8 && restrict_lanes != 16)
        return fail(ctx, MM_ERR_ARG, "restrict_lanes must be 0, 4, 8 or 16");
    ctx->tile_rows = ctx->P.tile_rows = rows_per_thread;
    ctx->restrict_lanes = ctx->P.restrict_lanes = restrict_lanes;
    return MM_OK;
}

int mm_set_magnetization(mm_ctx* ctx, const double* m) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!m) return fail(ctx, MM_ERR_ARG, "null m");
    return maybe_set_m(ctx, m);
}

int mm_set_magnetization_dev(mm_ctx* ctx, const double* m_dev) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!m_dev) return fail(ctx, MM_ERR_ARG, "null m");
    CK_CUDA(cudaMemcpyAsync(ctx->d_stage, m_dev, (size_t)ctx->n_nodes * 3 * sizeof(double),
                            cudaMemcpyDeviceToDevice, ctx->stream));
    return set_m_from_stage(ctx);
}

int mm_get_magnetization(mm_ctx* ctx, double* m_out) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!m_out) return fail(ctx, MM_ERR_ARG, "null output");
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    return copy_out3(ctx, ctx->P.X[ctx->h_state->cur], m_out);
}

int mm_get_magnetization_dev(mm_ctx* ctx, double* m_dev) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!m_dev) return fail(ctx, MM_ERR_ARG, "null output");
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    CK_CUDA(cudaMemsetAsync(m_dev, 0, (size_t)ctx->n_nodes * 3 * sizeof(double), ctx->stream));
    k_scatter3<<<nblk(ctx->nm), 256, 0, ctx->stream>>>(ctx->nm, ctx->d_mag_nodes, ctx->P.X[ctx->h_state->cur],
                                                        m_dev);
    CK_CUDA(cudaGetLastError());
    return MM_OK;
}

int mm_set_field(mm_ctx* ctx, const double mu0h[3]) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!mu0h) return fail(ctx, MM_ERR_ARG, "null field");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(mu0h[k])) return fail(ctx, MM_ERR_ARG, "non-finite field");
    k_set_field<<<1, 1, 0, ctx->stream>>>(ctx->d_state, mu0h[0] / (kMu0 * ctx->Mref),
                                          mu0h[1] / (kMu0 * ctx->Mref), mu0h[2] / (kMu0 * ctx->Mref));
    CK_CUDA(cudaGetLastError());
    for (int k = 0; k < 3; ++k) ctx->field_T[k] = mu0h[k];
    ctx->has_eval = false;
    return MM_OK;
}

int mm_minimize_async(mm_ctx* ctx, const mm_params* p) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if ((rc = check_params(ctx, p))) return rc;
    rc = launch_solver(ctx, mm::MODE_MINIMIZE, to_params(p));
    if (rc) return rc;
    ctx->has_eval = true;
    return MM_OK;
}

int mm_get_stats(mm_ctx* ctx, mm_stats* out) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    rc = finish(ctx);
    if (rc) return rc;
    if (out) fill_stats(ctx, out);
    return status_code(ctx->h_state->status);
}

int mm_minimize(mm_ctx* ctx, const mm_params* p, mm_stats* out) {
    int rc = mm_minimize_async(ctx, p);
    if (rc) return rc;
    rc = mm_get_stats(ctx, out);
    if (rc == MM_ERR_NONFINITE) fail(ctx, rc, "non-finite energy during minimisation");
    return rc;
}

int mm_energy(mm_ctx* ctx, const double* m, const mm_params* p, double* F, double terms[4]) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if ((rc = maybe_set_m(ctx, m))) return rc;
    if ((rc = eval_current(ctx, p))) return rc;
    const double EJ = kMu0 * ctx->Mref * ctx->Mref * 1e-27;
    if (F) *F = ctx->h_state->F * EJ;
    if (terms)
        for (int k = 0; k < 4; ++k) terms[k] = ctx->h_state->terms[k] * EJ;
    return MM_OK;
}

int mm_gradient(mm_ctx* ctx, const double* m, const mm_params* p, double* grad_out, int projected) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!grad_out) return fail(ctx, MM_ERR_ARG, "null output");
    if ((rc = maybe_set_m(ctx, m))) return rc;
    if ((rc = eval_current(ctx, p))) return rc;
    const int c = ctx->h_state->cur;
    return copy_out3(ctx, projected ? ctx->P.GP[c] : ctx->P.GR[c], grad_out);
}

int mm_get_potential(mm_ctx* ctx, double* phi_out) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!phi_out) return fail(ctx, MM_ERR_ARG, "null output");
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    CK_CUDA(cudaMemsetAsync(ctx->d_stage, 0, (size_t)ctx->n_nodes * sizeof(double), ctx->stream));
    k_scatter1<<<nblk(ctx->nphi), 256, 0, ctx->stream>>>(ctx->nphi, ctx->d_node_of_phi, ctx->d_ident, ctx->P.phi,
                                                          ctx->d_stage);
    CK_CUDA(cudaGetLastError());
    CK_CUDA(cudaMemcpyAsync(phi_out, ctx->d_stage, (size_t)ctx->n_nodes * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream));
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

int mm_precond_solve(mm_ctx* ctx, const mm_params* p, double* y_out, int64_t* steps) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!y_out) return fail(ctx, MM_ERR_ARG, "null output");
    if (!ctx->has_eval) return fail(ctx, MM_ERR_STATE, "no evaluation at the current state");
    if ((rc = check_params(ctx, p))) return rc;
    if ((rc = launch_solver(ctx, mm::MODE_PRECOND, to_params(p)))) return rc;
    if ((rc = finish(ctx))) return rc;
    if (steps) *steps = ctx->h_state->li;
    const int c = ctx->h_state->cur;
    return copy_out3(ctx, ctx->h_state->y_is_g ? ctx->P.GP[c] : ctx->P.isol, y_out);
}

int mm_hessian_apply(mm_ctx* ctx, const mm_params* p, const double* v, double* out) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!v || !out) return fail(ctx, MM_ERR_ARG, "null array");
    if (!ctx->has_eval) return fail(ctx, MM_ERR_STATE, "no evaluation at the current state");
    if ((rc = check_params(ctx, p))) return rc;
    CK_CUDA(cudaMemcpy(ctx->d_stage, v, (size_t)ctx->n_nodes * 3 * sizeof(double), cudaMemcpyHostToDevice));
    k_gather3<<<nblk(ctx->nm), 256, 0, ctx->stream>>>(ctx->nm, ctx->d_mag_nodes, ctx->d_stage, ctx->P.idir[0]);
    CK_CUDA(cudaGetLastError());
    if ((rc = launch_solver(ctx, mm::MODE_HESS, to_params(p)))) return rc;
    if ((rc = finish(ctx))) return rc;
    return copy_out3(ctx, ctx->P.ihd, out);
}

int mm_potential_matvec(mm_ctx* ctx, const double* v, double* out) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!v || !out) return fail(ctx, MM_ERR_ARG, "null array");
    CK_CUDA(cudaMemcpy(ctx->d_stage, v, (size_t)ctx->n_nodes * sizeof(double), cudaMemcpyHostToDevice));
    k_gather1<<<nblk(ctx->nphi), 256, 0, ctx->stream>>>(ctx->nphi, ctx->d_node_of_phi, ctx->d_ident,
                                                         ctx->d_stage, ctx->P.pdir[0]);
    CK_CUDA(cudaGetLastError());
    if ((rc = launch_solver(ctx, mm::MODE_KPHI, to_params(nullptr)))) return rc;
    if ((rc = finish(ctx))) return rc;
    CK_CUDA(cudaMemsetAsync(ctx->d_stage, 0, (size_t)ctx->n_nodes * sizeof(double), ctx->stream));
    k_scatter1<<<nblk(ctx->nphi), 256, 0, ctx->stream>>>(ctx->nphi, ctx->d_node_of_phi, ctx->d_ident, ctx->P.pq,
                                                          ctx->d_stage);
    CK_CUDA(cudaGetLastError());
    CK_CUDA(cudaMemcpyAsync(out, ctx->d_stage, (size_t)ctx->n_nodes * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->stream));
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

int mm_operator_apply(mm_ctx* ctx, int32_t op, const double* v, double* out) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (!v || !out) return fail(ctx, MM_ERR_ARG, "null array");
    if (op != MM_OP_DIV && op != MM_OP_DIVT && op != MM_OP_LOCAL) return fail(ctx, MM_ERR_ARG, "unknown operator %d", op);
    const size_t N = (size_t)ctx->n_nodes;
    if (op == MM_OP_DIVT) {
        CK_CUDA(cudaMemcpy(ctx->d_stage, v, N * sizeof(double), cudaMemcpyHostToDevice));
        k_gather1<<<nblk(ctx->nphi), 256, 0, ctx->stream>>>(ctx->nphi, ctx->d_node_of_phi, ctx->d_ident,
                                                             ctx->d_stage, ctx->P.pdir[0]);
    } else {
        CK_CUDA(cudaMemcpy(ctx->d_stage, v, 3 * N * sizeof(double), cudaMemcpyHostToDevice));
        k_gather3<<<nblk(ctx->nm), 256, 0, ctx->stream>>>(ctx->nm, ctx->d_mag_nodes, ctx->d_stage, ctx->P.idir[0]);
    }
    CK_CUDA(cudaGetLastError());
    const int mode = (op == MM_OP_DIV) ? mm::MODE_DIV : (op == MM_OP_DIVT) ? mm::MODE_DIVT : mm::MODE_LOCAL;
    if ((rc = launch_solver(ctx, mode, to_params(nullptr)))) return rc;
    if ((rc = finish(ctx))) return rc;
    if (op != MM_OP_DIV) return copy_out3(ctx, ctx->P.ihd, out);
    CK_CUDA(cudaMemsetAsync(ctx->d_stage, 0, N * sizeof(double), ctx->stream));
    k_scatter1<<<nblk(ctx->nphi), 256, 0, ctx->stream>>>(ctx->nphi, ctx->d_node_of_phi, ctx->d_ident, ctx->P.pq,
                                                          ctx->d_stage);
    CK_CUDA(cudaGetLastError());
    CK_CUDA(cudaMemcpyAsync(out, ctx->d_stage, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

int mm_demag_curve(mm_ctx* ctx, int64_t n_fields, const double* fields, const mm_params* p, mm_stats* stats_out) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (n_fields < 0 || (n_fields > 0 && !fields)) return fail(ctx, MM_ERR_ARG, "bad field list");
    if ((rc = check_params(ctx, p))) return rc;
    int first = MM_OK;
    for (int64_t k = 0; k < n_fields; ++k) {
        if ((rc = mm_set_field(ctx, fields + 3 * k))) return rc;
        mm_stats st;
        rc = mm_minimize(ctx, p, &st);
        if (rc == MM_ERR_DEVICE_TIMEOUT || rc == MM_ERR_CUDA) return rc;
        if (stats_out) stats_out[k] = st;
        if (first == MM_OK && rc != MM_OK) first = rc;
    }
    return first;
}

int mm_autotune_jmax(mm_ctx* ctx, const mm_params* p, int64_t n_fields, const double* fields,
                     const int32_t* candidates, int32_t n_candidates, int32_t* best_jmax, double* ms_out) {
    int rc = need_mesh(ctx);
    if (rc) return rc;
    if (n_fields < 1 || !fields || !candidates || n_candidates < 1 || !best_jmax)
        return fail(ctx, MM_ERR_ARG, "bad autotune arguments");
    for (int32_t c = 0; c < n_candidates; ++c)
        if (candidates[c] < 0) return fail(ctx, MM_ERR_ARG, "candidate j_max must be >= 0");
    if ((rc = check_params(ctx, p))) return rc;
    mm_params q;
    if (p) q = *p;
    else mm_default_params(&q);
    // the state every trial starts from: m and potential of the current
    // slot, the applied field
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    const int cur = ctx->h_state->cur;
    const size_t v3 = 3 * (size_t)ctx->nm, np = (size_t)ctx->nphi;
    double* save = nullptr;
    CK_CUDA(cudaMalloc(&save, (v3 + 2 * np) * sizeof(double)));
    auto restore = [&]() -> int {
        CK_CUDA(cudaMemcpyAsync(ctx->P.X[cur], save, v3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CK_CUDA(cudaMemcpyAsync(ctx->P.PHI[cur], save + v3, np * sizeof(double), cudaMemcpyDeviceToDevice,
                                ctx->stream));
        CK_CUDA(cudaMemcpyAsync(ctx->P.phi, save + v3 + np, np * sizeof(double), cudaMemcpyDeviceToDevice,
                                ctx->stream));
        k_set_cur<<<1, 1, 0, ctx->stream>>>(ctx->d_state, cur);
        CK_CUDA(cudaGetLastError());
        ctx->has_eval = false;
        return MM_OK;
    };
    CK_CUDA(cudaMemcpyAsync(save, ctx->P.X[cur], v3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CK_CUDA(cudaMemcpyAsync(save + v3, ctx->P.PHI[cur], np * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CK_CUDA(cudaMemcpyAsync(save + v3 + np, ctx->P.phi, np * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    const double f0[3] = {ctx->field_T[0], ctx->field_T[1], ctx->field_T[2]};
    double best = -1.0;
    int first_err = MM_OK;
    for (int32_t c = 0; c < n_candidates && first_err == MM_OK; ++c) {
        q.jmax = candidates[c];
        double tot = 0.0;
        for (int64_t k = 0; k < n_fields; ++k) {
            if ((rc = mm_set_field(ctx, fields + 3 * k))) break;
            if ((rc = mm_minimize_async(ctx, &q))) break;
            mm_stats st;
            rc = mm_get_stats(ctx, &st);
            if (rc < 0) break;
            double ms = 0.0;
            if ((rc = mm_last_kernel_ms(ctx, &ms))) break;
            tot += ms;
            rc = MM_OK;
        }
        if (rc < 0) first_err = rc;
        if (rc >= 0 && (best < 0.0 || tot < best)) {
            best = tot;
            *best_jmax = candidates[c];
        }
        if (ms_out) ms_out[c] = tot;
        const int rr = restore();
        if (rr && first_err == MM_OK) first_err = rr;
    }
    if (first_err == MM_OK) first_err = mm_set_field(ctx, f0);
    CK_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->h_state->cur = cur;              // the host mirror of the restored slot
    cudaFree(save);
    return first_err;
}

int mm_last_kernel_ms(mm_ctx* ctx, double* ms) {
    if (!ctx || !ms) return MM_ERR_ARG;
    if (!ctx->timed) return fail(ctx, MM_ERR_STATE, "no kernel launched yet");
    CK_CUDA(cudaEventSynchronize(ctx->ev1));
    float f = 0.f;
    CK_CUDA(cudaEventElapsedTime(&f, ctx->ev0, ctx->ev1));
    *ms = f;
    return MM_OK;
}

}  // extern "C"
