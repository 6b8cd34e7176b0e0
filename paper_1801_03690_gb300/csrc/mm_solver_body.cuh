// Persistent solver kernel: Algorithm 4 (projected preconditioned NCG) with
// its two inner solvers (Algorithm 1 on the scalar-potential stiffness and
// on the approximate Hessian of Eq. precond), run entirely on the device.
//
// One cooperative launch covers a whole minimisation.  The blocks form a
// team that moves through phases separated by team barriers; every phase is
// a grid-stride pass over rows (one thread per SELL-32 row) that also writes
// per-block partial sums.  After a barrier every block reduces the same
// partials in the same fixed order, so all blocks hold bit-identical scalars
// and take the same branch at every decision (potential-solve convergence,
// li1-li3, line-search branches, beta*ZA, t1-t3) without host round trips or
// atomics on floating-point data.  Barrier waits are bounded: a wait that
// runs out sets the device error flag and every block leaves the kernel.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr unsigned long long kBarrierTimeoutNs = 5000000000ull;  // 5 s per wait
constexpr int kWarps = MM_BLOCK / 32;

struct Team {
    int nb;
    int rank;
    unsigned long long* count;   // arrival counter (barrier words [0..1])
    int* err;
    double* part;
    int epoch;
    bool dead;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Team barrier with a bounded wait.  The arrival counter is 64-bit and only
// grows (zeroed by the host before each launch): a block's k-th barrier is
// complete once the counter reaches k * nb, so the last arriver publishes
// completion with its own increment and no reset or second word is needed
// (measured on GB300: 1.9 us per empty barrier with a reset counter and a
// generation word).  The fences make each block's writes before the barrier
// visible to every block after it.
__device__ bool team_sync(Team& t) {
    __shared__ int s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* verr = t.err;
        int e = *verr;
        if (e == 0) {
            const unsigned long long nb = (unsigned long long)t.nb;
            __threadfence();
            const unsigned long long old = atomicAdd(t.count, 1ull);
            const unsigned long long target = (old / nb + 1ull) * nb;
            if (old + 1ull != target) {
                volatile unsigned long long* vc = t.count;
                const unsigned long long t0 = global_ns();
                while (*vc < target) {
                    if (*verr) break;
                    __nanosleep(32);
                    if (global_ns() - t0 > kBarrierTimeoutNs) {
                        atomicCAS(t.err, 0, (int)ST_TIMEOUT);
                        break;
                    }
                }
            }
            __threadfence();
            e = *verr;
        }
        s_err = e;
    }
    __syncthreads();
    t.dead = (s_err != 0);
    return !t.dead;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Reduce NS sums and NX maxima over the team.  Deterministic: fixed order
// within warps (shfl_down tree, lane 0), across warps (ascending) and across
// blocks (ascending strided accumulation, then the same block tree).
template <typename AT>
__device__ __forceinline__ AT warp_sum_t(AT v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <typename AT>
__device__ __forceinline__ AT warp_max_t(AT v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// AT is the type of the per-thread and per-warp accumulation (float for the
// FP32 phases, whose sums are all of positive terms); the combination across
// warps and blocks is always FP64.
template <int NS, int NX, typename AT = double>
__device__ bool team_reduce(Team& t, AT (&s)[NS > 0 ? NS : 1], AT (&x)[NX > 0 ? NX : 1]) {
    static_assert(NS + NX <= MM_MAXRED, "too many reduction values");
    __shared__ double sh[MM_MAXRED][kWarps];
    __shared__ double res[MM_MAXRED];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        AT v = warp_sum_t<AT>(s[k]);
        if (lane == 0) sh[k][warp] = (double)v;
    }
#pragma unroll
    for (int k = 0; k < NX; ++k) {
        AT v = warp_max_t<AT>(x[k]);
        if (lane == 0) sh[NS + k][warp] = (double)v;
    }
    __syncthreads();
    double* part = t.part + (size_t)(t.epoch & 1) * MM_MAXRED * t.nb;
    if (threadIdx.x < NS + NX) {
        const int k = threadIdx.x;
        double a = sh[k][0];
        for (int w = 1; w < kWarps; ++w) a = (k < NS) ? a + sh[k][w] : fmax(a, sh[k][w]);
        part[(size_t)k * t.nb + t.rank] = a;
    }
    t.epoch++;
    if (!team_sync(t)) return false;
    // every block folds all partials identically
#pragma unroll
    for (int k = 0; k < NS + NX; ++k) {
        const double* pk = part + (size_t)k * t.nb;
        double a = (k < NS) ? 0.0 : 0.0;
        for (int j = threadIdx.x; j < t.nb; j += MM_BLOCK) a = (k < NS) ? a + pk[j] : fmax(a, pk[j]);
        a = (k < NS) ? warp_sum(a) : warp_max(a);
        if (lane == 0) sh[k][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < NS + NX) {
        const int k = threadIdx.x;
        double a = sh[k][0];
        for (int w = 1; w < kWarps; ++w) a = (k < NS) ? a + sh[k][w] : fmax(a, sh[k][w]);
        res[k] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NS; ++k) s[k] = (AT)res[k];
#pragma unroll
    for (int k = 0; k < NX; ++k) x[k] = (AT)res[NS + k];
    __syncthreads();
    return true;
}

// Team sums accumulated in FP32 per thread and warp, returned in FP64.
template <int NS>
__device__ bool team_sum_f32(Team& t, float (&s)[NS], double (&out)[NS]) {
    __shared__ double sh[MM_MAXRED][kWarps];
    __shared__ double res[MM_MAXRED];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const float v = warp_sum_t<float>(s[k]);
        if (lane == 0) sh[k][warp] = (double)v;
    }
    __syncthreads();
    double* part = t.part + (size_t)(t.epoch & 1) * MM_MAXRED * t.nb;
    if (threadIdx.x < NS) {
        const int k = threadIdx.x;
        double a = sh[k][0];
        for (int w = 1; w < kWarps; ++w) a += sh[k][w];
        part[(size_t)k * t.nb + t.rank] = a;
    }
    t.epoch++;
    if (!team_sync(t)) return false;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const double* pk = part + (size_t)k * t.nb;
        double a = 0.0;
        for (int j = threadIdx.x; j < t.nb; j += MM_BLOCK) a += pk[j];
        a = warp_sum(a);
        if (lane == 0) sh[k][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < NS) {
        const int k = threadIdx.x;
        double a = sh[k][0];
        for (int w = 1; w < kWarps; ++w) a += sh[k][w];
        res[k] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NS; ++k) out[k] = res[k];
    __syncthreads();
    return true;
}

struct Row {
    long long base;
    int width;
};

__device__ __forceinline__ Row sell_row(const long long* sptr, int r) {
    const int s = r >> 5;
    const long long b = sptr[s];
    return {b + (r & 31), (int)((sptr[s + 1] - b) >> 5)};
}

#define ROWS(r, n) for (int r = t.rank * MM_BLOCK + (int)threadIdx.x; r < (n); r += t.nb * MM_BLOCK)
// Row dot products over a SELL-32 row.  All column indices and values of a
// chunk are loaded before any gather, so each thread keeps a whole row's
// worth of independent loads in flight: measured on GB300 this lifts an FP32
// SpMV from 3.8 to 6.6 TB/s inside the persistent kernel.  The matrix
// entries are read once per product, so they are loaded with the
// evict-first (streaming) policy, which leaves L2 to the gathered vectors
// (+1.5% NCG iterations/s on the 8.7 M-unknown polycrystal).
// Lanes past the row's width read x[pad] (pad = r for square matrices, 0
// for rectangular ones whose row index may exceed the columns).
template <int CH, typename T, typename VT, typename XT>
__device__ __forceinline__ T sell_dot(const long long* __restrict__ sptr, const int* __restrict__ col,
                                      const VT* __restrict__ val, const XT* x, int r, int pad) {
    const Row A = sell_row(sptr, r);
    T s = T(0);
    for (int k0 = 0; k0 < A.width; k0 += CH) {
        int c[CH];
        VT v[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const bool ok = k0 + u < A.width;
            const long long e = A.base + 32ll * (k0 + u);
            c[u] = ok ? __ldcs(col + e) : pad;
            v[u] = ok ? __ldcs(val + e) : VT(0);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) s += (T)v[u] * (T)x[c[u]];
    }
    return s;
}

template <int CH, typename T, typename VT, typename XT>
__device__ __forceinline__ T sell_dot(const long long* __restrict__ sptr, const int* __restrict__ col,
                                      const VT* __restrict__ val, const XT* x, int r) {
    return sell_dot<CH, T>(sptr, col, val, x, r, r);
}

// Same for a scalar matrix applied to a SoA 3-vector (stride n); T the
// type of the sums and of the values (FP64, or FP32 in the precision form's
// preconditioner).
template <int CH, typename T>
__device__ __forceinline__ void sell_dot3(const long long* __restrict__ sptr, const int* __restrict__ col,
                                          const T* __restrict__ val, const T* x, int n, int r,
                                          T& s0, T& s1, T& s2) {
    const Row A = sell_row(sptr, r);
    s0 = s1 = s2 = T(0);
    for (int k0 = 0; k0 < A.width; k0 += CH) {
        int c[CH];
        T v[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const bool ok = k0 + u < A.width;
            const long long e = A.base + 32ll * (k0 + u);
            c[u] = ok ? __ldg(col + e) : r;
            v[u] = ok ? __ldg(val + e) : T(0);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            s0 += v[u] * x[c[u]];
            s1 += v[u] * x[n + c[u]];
            s2 += v[u] * x[2 * n + c[u]];
        }
    }
}

// Two SELL-32 rows r0 and r1 = r0 + team stride (two: r1 exists) per thread,
// CH entries of both rows loaded before any gather: twice the loads in
// flight of the one-row form at the register cost of CH = 16.  Used by the
// FP32 direction step and the level-0 products of the multigrid cycle,
// whose rows hold a handful of entries.  Lanes past a row's width read
// x[pad].
template <int CH, typename VT>
__device__ __forceinline__ void sell_dot_2rows(const long long* __restrict__ sptr, const int* __restrict__ col,
                                               const VT* __restrict__ val, const VT* x, int r0, int r1,
                                               bool two, int pad, VT& s0, VT& s1) {
    const Row A = sell_row(sptr, r0);
    const Row B = two ? sell_row(sptr, r1) : Row{0, 0};
    s0 = VT(0);
    s1 = VT(0);
    const int w = A.width > B.width ? A.width : B.width;
    for (int k0 = 0; k0 < w; k0 += CH) {
        int c0[CH], c1[CH];
        VT v0[CH], v1[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const bool ok0 = k0 + u < A.width, ok1 = k0 + u < B.width;
            c0[u] = ok0 ? __ldcs(col + A.base + 32ll * (k0 + u)) : pad;
            v0[u] = ok0 ? __ldcs(val + A.base + 32ll * (k0 + u)) : VT(0);
            c1[u] = ok1 ? __ldcs(col + B.base + 32ll * (k0 + u)) : pad;
            v1[u] = ok1 ? __ldcs(val + B.base + 32ll * (k0 + u)) : VT(0);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            s0 += v0[u] * x[c0[u]];
            s1 += v1[u] * x[c1[u]];
        }
    }
}

// The offset table of the slice of row r (MM_NO_TAB in entry 0: the slice
// keeps its column array), two 16-byte loads that every lane of the warp
// makes at the same address.
struct SliceTab {
    int d[8];
};
__device__ __forceinline__ SliceTab slice_tab(const int* __restrict__ tab, int r) {
    const int4* t4 = reinterpret_cast<const int4*>(tab) + 2 * (r >> 5);
    const int4 a = __ldg(t4), b = __ldg(t4 + 1);
    return {{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w}};
}

// sell_dot_2rows for the FP32 K_phi layout with slice offset tables: when
// both rows' slices have a table (at most 8 entries per row), entry u of row
// r is column r + tab[u] and only the values are loaded; otherwise both rows
// go through sell_dot_2rows on the layout's columns.  The entries of a table
// slice are the row's couplings in column order with zeros for the offsets
// it lacks, so the sums are those of the plain layout.  Square matrices
// only (lanes past a row's width read x[r0]).
__device__ __forceinline__ void sell_dot_2rows_tab(const long long* __restrict__ sptr, const int* __restrict__ col,
                                                   const float* __restrict__ val, const int* __restrict__ tab,
                                                   const float* x, int r0, int r1, bool two, float& s0, float& s1) {
    const SliceTab ta = slice_tab(tab, r0);
    const SliceTab tb = slice_tab(tab, two ? r1 : r0);
    if (ta.d[0] == MM_NO_TAB || tb.d[0] == MM_NO_TAB) {
        sell_dot_2rows<8>(sptr, col, val, x, r0, r1, two, r0, s0, s1);
        return;
    }
    const Row A = sell_row(sptr, r0);
    const Row B = two ? sell_row(sptr, r1) : Row{0, 0};
    float v0[8], v1[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        v0[u] = u < A.width ? __ldcs(val + A.base + 32ll * u) : 0.0f;
        v1[u] = u < B.width ? __ldcs(val + B.base + 32ll * u) : 0.0f;
    }
    s0 = 0.0f;
    s1 = 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        s0 += v0[u] * x[u < A.width ? r0 + ta.d[u] : r0];
        s1 += v1[u] * x[u < B.width ? r1 + tb.d[u] : r0];
    }
}

// One row of the same layout (sell_dot's one-row form, 16 entries per chunk).
__device__ __forceinline__ float sell_dot_tab(const long long* __restrict__ sptr, const int* __restrict__ col,
                                              const float* __restrict__ val, const int* __restrict__ tab,
                                              const float* x, int r) {
    const SliceTab ta = slice_tab(tab, r);
    if (ta.d[0] == MM_NO_TAB) return sell_dot<16, float>(sptr, col, val, x, r, r);
    const Row A = sell_row(sptr, r);
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = u < A.width ? __ldcs(val + A.base + 32ll * u) : 0.0f;
    float s = 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u] * x[u < A.width ? r + ta.d[u] : r];
    return s;
}

// Grid-stride loop over row pairs (r, r2 = r + team stride); two: r2 < n.
#define ROWS2(r, r2, two, n)                                                                     \
    for (int r = t.rank * MM_BLOCK + (int)threadIdx.x, r2 = 0; r < (n); r += 2 * t.nb * MM_BLOCK) \
        if (const bool two = ((r2 = r + t.nb * MM_BLOCK) < (n)); true)

// The FP32 products of level 0 (K_phi and the smoothed prolongation) over the
// team's rows in the tile shape P.tile_rows selects; f(r, s, v) takes row r,
// its sum s and v = pre(r), the row's vector operands, which pre loads before
// the product's loads are issued: the vector loads then overlap the matrix
// loads and the gathers instead of following them.  Both shapes visit a
// thread's rows in the same order (r, r + stride, r + 2 stride, ...), so
// per-thread sums f accumulates come out in the same order too.  tab: the
// slice offset tables of the FP32 K_phi (nullptr for other matrices).
// pad_self: lanes past a row's width gather x[r] (square matrices) rather
// than x[0].
template <class Pre, class F>
__device__ __forceinline__ void level0_products(const Problem& P, const Team& t, const long long* __restrict__ sptr,
                                                const int* __restrict__ col, const float* __restrict__ val,
                                                const int* __restrict__ tab, const float* x, int n, bool pad_self,
                                                Pre pre, F f) {
    if (P.tile_rows != 1) {
        ROWS2(r, r2, two, n) {
            const auto v0 = pre(r);
            const auto v1 = pre(two ? r2 : r);
            float s0, s1;
            if (tab) sell_dot_2rows_tab(sptr, col, val, tab, x, r, r2, two, s0, s1);
            else sell_dot_2rows<8>(sptr, col, val, x, r, r2, two, pad_self ? r : 0, s0, s1);
            f(r, s0, v0);
            if (two) f(r2, s1, v1);
        }
    } else {
        ROWS(r, n) {
            const auto v0 = pre(r);
            f(r, tab ? sell_dot_tab(sptr, col, val, tab, x, r) : sell_dot<16, float>(sptr, col, val, x, r, pad_self ? r : 0),
              v0);
        }
    }
}

// ---- row kernels of the three operators of Eq. (energy) on the magnetic
// graph, shared by the solver phases and the operator entry point.

// (D x)_p of a magnetic row p (Sec. 3.1: the right-hand side of the
// potential equation), x a SoA 3-vector over the magnetic nodes.
__device__ __forceinline__ double row_div(const Problem& P, const double* x, int p) {
    const int nm = P.nm;
    const long long nz = P.nnzm;
    const Row mr = sell_row(P.m_sptr, p);
    double bp = 0.0;
    for (int k0 = 0; k0 < mr.width; k0 += 8) {
        int c[8];
        double b0[8], b1[8], b2[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool ok = k0 + u < mr.width;
            const long long e = mr.base + 32ll * (k0 + u);
            c[u] = ok ? __ldg(P.m_col + e) : p;
            b0[u] = ok ? __ldg(P.B + e) : 0.0;
            b1[u] = ok ? __ldg(P.B + nz + e) : 0.0;
            b2[u] = ok ? __ldg(P.B + 2 * nz + e) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) bp += b0[u] * x[c[u]] + b1[u] * x[nm + c[u]] + b2[u] * x[2 * nm + c[u]];
    }
    return bp;
}

// (D^T phi)_i of a magnetic node i (the magnetostatic part of the gradient).
__device__ __forceinline__ void row_divT(const Problem& P, const double* phi, int i, double& t0, double& t1,
                                         double& t2) {
    const long long nz = P.nnzm;
    const Row rw = sell_row(P.m_sptr, i);
    t0 = t1 = t2 = 0.0;
    for (int k0 = 0; k0 < rw.width; k0 += 8) {
        int c[8];
        double q0[8], q1[8], q2[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool ok = k0 + u < rw.width;
            const long long e = rw.base + 32ll * (k0 + u);
            c[u] = ok ? __ldg(P.m_col + e) : i;
            q0[u] = ok ? __ldg(P.G + e) : 0.0;
            q1[u] = ok ? __ldg(P.G + nz + e) : 0.0;
            q2[u] = ok ? __ldg(P.G + 2 * nz + e) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const double ph = phi[c[u]];
            t0 += q0[u] * ph;
            t1 += q1[u] * ph;
            t2 += q2[u] * ph;
        }
    }
}

// The local operators at node i: c = K_A x (exchange stiffness on each
// component; C_A x = 2 c) and a = C_K x (the lumped anisotropy block).
__device__ __forceinline__ void row_local(const Problem& P, const double* x, int i, double& c0, double& c1,
                                          double& c2, double& a0, double& a1, double& a2) {
    const int nm = P.nm;
    sell_dot3<8>(P.m_sptr, P.m_col, P.KA, x, nm, i, c0, c1, c2);
    const double x0 = x[i], x1 = x[nm + i], x2 = x[2 * nm + i];
    const double kxx = P.CK[i], kxy = P.CK[nm + i], kxz = P.CK[2 * nm + i];
    const double kyy = P.CK[3 * nm + i], kyz = P.CK[4 * nm + i], kzz = P.CK[5 * nm + i];
    a0 = kxx * x0 + kxy * x1 + kxz * x2;
    a1 = kxy * x0 + kyy * x1 + kyz * x2;
    a2 = kxz * x0 + kyz * x1 + kzz * x2;
}

struct SlotScalars {
    double F, terms[4], gmax, dphi, xdiff, xmax, M[3];
};

struct Ctx {
    const Problem* P;
    Team t;
    long long evals, nli, li, mi, ls_extra, mr;
    long long li2, li2_first, restarts, steepest;
    double h[3];
    SlotScalars sl[MM_NSLOT];
    int y_is_g;
    double ptol;             // relative residual the potential solves stop at
    double gy_prev;          // g_j . y_j of the last direction (beta*FR, beta*PRP)
};

// ---------------------------------------------------------------- phases

// x_s = N(x_c + a d), |x_c + a d| kept for Eq. (opt2); max|x_s - x_c|, max|x_s|.
__device__ bool ph_trial(Ctx& C, int c, int s, double a) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    double mx[2] = {0.0, 0.0};
    double dummy[1] = {0.0};
    const double* xc = P.X[c];
    double* xs = P.X[s];
    ROWS(i, nm) {
        double u0 = xc[i] + a * P.d[i];
        double u1 = xc[nm + i] + a * P.d[nm + i];
        double u2 = xc[2 * nm + i] + a * P.d[2 * nm + i];
        double n = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
        double v0 = u0 / n, v1 = u1 / n, v2 = u2 / n;
        xs[i] = v0;
        xs[nm + i] = v1;
        xs[2 * nm + i] = v2;
        P.unorm[i] = n;
        mx[0] = fmax(mx[0], fmax(fabs(v0 - xc[i]), fmax(fabs(v1 - xc[nm + i]), fabs(v2 - xc[2 * nm + i]))));
        mx[1] = fmax(mx[1], fmax(fabs(v0), fmax(fabs(v1), fabs(v2))));
    }
    if (!team_reduce<0, 2>(t, dummy, mx)) return false;
    C.sl[s].xdiff = mx[0];
    C.sl[s].xmax = mx[1];
    return true;
}

// Potential-solve set-up: rhs = D x_s on the magnetic rows, r = rhs - K phi,
// z = diag(K)^-1 r.  Sums: |rhs|^2, r.z, |r|^2.
__device__ bool ph_pinit(Ctx& C, int s, double& bb, double& rz, double& rr) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    const double* x = P.X[s];
    double acc[3] = {0.0, 0.0, 0.0};
    double dummy[1] = {0.0};
    ROWS(p, P.nphi) {
        const double kphi = sell_dot<8, double>(P.p_sptr, P.p_col, P.Kp, P.phi, p);
        double bp = 0.0;
        if (p < nm) {
            bp = row_div(P, x, p);
            P.rhs[p] = bp;
        }
        const double r = bp - kphi;
        const double z = r * P.dinvP[p];
        P.pres[p] = r;
        P.pprec[p] = z;
        acc[0] += bp * bp;
        acc[1] += r * z;
        acc[2] += r * r;
    }
    if (!team_reduce<3, 0>(t, acc, dummy)) return false;
    bb = acc[0];
    rz = acc[1];
    rr = acc[2];
    return true;
}

// Plain product q = K v (no reduction).
__device__ bool ph_pmatvec(Ctx& C, const double* v, double* q) {
    const Problem& P = *C.P;
    Team& t = C.t;
    ROWS(p, P.nphi) q[p] = sell_dot<8, double>(P.p_sptr, P.p_col, P.Kp, v, p);
    return team_sync(t);
}

// CG direction step of Algorithm 1 with the product formed by recurrence:
// w = K z, d = z + beta d, q = w + beta q (= K d), in place.  Sum: d . q.
__device__ bool ph_pdirection(Ctx& C, const double* z, double beta, double* d, double* q, double& dq) {
    const Problem& P = *C.P;
    Team& t = C.t;
    double acc[1] = {0.0};
    double dummy[1] = {0.0};
    const bool first = (beta == 0.0);
    ROWS(p, P.nphi) {
        const double s = sell_dot<8, double>(P.p_sptr, P.p_col, P.Kp, z, p);
        const double dn = first ? z[p] : z[p] + beta * d[p];
        const double qn = first ? s : s + beta * q[p];
        d[p] = dn;
        q[p] = qn;
        acc[0] += dn * qn;
    }
    if (!team_reduce<1, 0>(t, acc, dummy)) return false;
    dq = acc[0];
    return true;
}

// phi += a v; r -= a q; z = diag^-1 r.  Sums: r.z, |r|^2.
__device__ bool ph_pupdate(Ctx& C, const double* v, double a, double& rz, double& rr) {
    const Problem& P = *C.P;
    Team& t = C.t;
    double acc[2] = {0.0, 0.0};
    double dummy[1] = {0.0};
    ROWS(p, P.nphi) {
        P.phi[p] += a * v[p];
        const double r = P.pres[p] - a * P.pq[p];
        const double z = r * P.dinvP[p];
        P.pres[p] = r;
        P.pprec[p] = z;
        acc[0] += r * z;
        acc[1] += r * r;
    }
    if (!team_reduce<2, 0>(t, acc, dummy)) return false;
    rz = acc[0];
    rr = acc[1];
    return true;
}

__device__ bool ph_pzero(Ctx& C) {
    const Problem& P = *C.P;
    Team& t = C.t;
    ROWS(p, P.nphi) {
        P.phi[p] = 0.0;
        P.pres[p] = 0.0;
    }
    return team_sync(t);
}

// ---- precision form of the potential solve: the correction equation
// K delta = r (r the FP64 residual) is solved by Algorithm 1 in FP32 (FP32
// operator, vectors and products; FP64 reductions); then phi += delta and
// r -= K delta in FP64 (iterative refinement of the FP64 residual).

// Compensated FP32 accumulation (Ogita, Rump and Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26 (2005), algorithm Dot2): the
// rounding error of every product (by FMA) and of every addition (by the
// two-sum transformation) is collected in a second FP32 word, so the result
// is as accurate as if computed in twice the working precision.  The
// restriction rows of the smoothed aggregates sum a few hundred terms that
// largely cancel; their rounding would otherwise enter the coarse
// correction amplified by the coarse inverse.
struct Dot2 {
    float p, s;
};

// (The _rn intrinsics keep the compiler from contracting the transformations
// into FMAs, which would break their exactness.)
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
    const float x = __fadd_rn(a, b);
    const float z = __fsub_rn(x, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(x, z)), __fsub_rn(b, z));
    return x;
}

__device__ __forceinline__ void dot2_add(Dot2& d, float a, float b) {
    const float h = __fmul_rn(a, b);
    const float r = __fmaf_rn(a, b, -h);     // exact: a b = h + r
    float q;
    d.p = two_sum(d.p, h, q);
    d.s = __fadd_rn(d.s, __fadd_rn(q, r));
}

__device__ __forceinline__ void dot2_merge(Dot2& d, float p, float s) {
    float q;
    d.p = two_sum(d.p, p, q);
    d.s = __fadd_rn(d.s, __fadd_rn(s, q));
}

// The dot product of CSR row `row` (< 0: an empty row) with x, computed by a
// group of G consecutive lanes (G divides 32): lane gl of the group takes
// entries gl, gl + G, ..., CH per pass with all of a pass's loads issued
// before any gather, accumulates them compensated, and the group combines
// its lanes with a G-lane xor reduction (every lane of the warp takes part).
template <int G, int CH, class XF>
__device__ __forceinline__ float group_csr_dot2(const long long* __restrict__ ptr, const int* __restrict__ col,
                                                const float* __restrict__ val, XF x, int row, int gl) {
    const long long b = row >= 0 ? ptr[row] : 0, e = row >= 0 ? ptr[row + 1] : 0;
    Dot2 s = {0.0f, 0.0f};
    for (long long o = b + gl; o < e; o += (long long)G * CH) {
        int c[CH];
        float v[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const long long k = o + (long long)G * u;
            const bool ok = k < e;
            c[u] = ok ? __ldcs(col + k) : 0;
            v[u] = ok ? __ldcs(val + k) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) dot2_add(s, v[u], x(c[u]));
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const float p = __shfl_xor_sync(0xffffffffu, s.p, off);
        const float q = __shfl_xor_sync(0xffffffffu, s.s, off);
        dot2_merge(s, p, q);
    }
    return s.p + s.s;
}

// ---- smoothed-aggregation multigrid V-cycle (the FP32 solve's
// preconditioner when a hierarchy exists and prm.amg is set); operators as
// in struct Level.  A down phase computes rpre = b - A x on the rows of its
// level (one thread per row), then, after a team barrier, b_{l+1} = P^T rpre
// and x_{l+1} = omega D^-1 b_{l+1} on the rows of the next level (a group of
// lanes per row).

// Restriction rows of a down phase: b_{l+1} = P^T r with r(j) given by bx,
// x_{l+1} = omega D^-1 b_{l+1}.  A group of G lanes per coarse row, so a
// warp works on 32 / G rows at once: at the fine end the rows of P^T hold
// tens of entries (2.9 per fine row on the lattice meshes), and a whole warp
// per row spent its time in the 5-level shuffle reduction.
template <int G, class XF>
__device__ __forceinline__ void amg_restrict_g(const Problem& P, const Team& t, const Level& V, int l, XF bx) {
    constexpr int RPW = 32 / G;
    const bool last = (l + 1 == P.nlev);
    float* bn = last ? P.bco : P.lev[l + 1].b;
    float* xn = last ? nullptr : P.lev[l + 1].x;
    const float* dn = last ? nullptr : P.lev[l + 1].dinv;
    const float on = last ? 0.0f : P.lev[l + 1].omega;
    const int lane = threadIdx.x & 31, wpb = MM_BLOCK / 32, nw = t.nb * wpb;
    const int gw = t.rank * wpb + (int)(threadIdx.x >> 5), grp = lane / G, gl = lane % G;
    for (int I0 = gw * RPW; I0 < V.nc; I0 += nw * RPW) {
        const int I = I0 + grp;
        const float s = group_csr_dot2<G, 12>(V.t_ptr, V.t_col, V.t_val, bx, I < V.nc ? I : -1, gl);
        if (gl == 0 && I < V.nc) {
            bn[I] = s;
            if (!last) xn[I] = on * dn[I] * s;
        }
    }
}

// Levels with few, long restriction rows (the coarse end of the hierarchy:
// hundreds of entries per row, a few hundred rows) take a whole warp per
// row, the others a group of P.restrict_lanes lanes, 8 by default (measured
// on the 8.7 M-unknown polycrystal: 8 lanes 190 us, 4 lanes 211, 16 lanes
// 225 for the level-0 down phase).
template <class XF>
__device__ __forceinline__ void amg_restrict(const Problem& P, const Team& t, const Level& V, int l, XF bx) {
    if (V.wide) amg_restrict_g<32>(P, t, V, l, bx);
    else if (P.restrict_lanes == 4) amg_restrict_g<4>(P, t, V, l, bx);
    else if (P.restrict_lanes == 16) amg_restrict_g<16>(P, t, V, l, bx);
    else amg_restrict_g<8>(P, t, V, l, bx);
}

// Down phase of level l; at level 0, b is the FP32 residual and x = omega
// D^-1 b has been written with it by the update step.  The pre-smoothed
// residual rpre is restricted after a team barrier with P^T, which holds
// half the entries of U^T (U^T b, the same vector, needs no barrier:
// measured on the 8.7 M-unknown polycrystal, the U^T restriction took 205
// of the phase's 323 us).
// rpre = b - A x on the rows of level 0 (K_phi, a handful of entries per
// row), a function of its own so that its registers are allocated apart
// from the restriction's.
__device__ __noinline__ void amg_down0_rows(const Problem& P, const Team& t) {
    const Level& V = P.lev[0];
    const float* b = P.pres32;
    level0_products(P, t, V.sptr, V.col, V.val, V.tab, P.amg_x0, V.n, true, [&](int r) { return b[r]; },
                    [&](int r, float s, float br) { V.rpre[r] = br - s; });
}

__device__ __noinline__ bool ph_amg_down(Ctx& C, int l) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const Level& V = P.lev[l];
    if (l == 0) {
        amg_down0_rows(P, t);
    } else {
        ROWS(r, V.n) V.rpre[r] = V.b[r] - sell_dot<16, float>(V.sptr, V.col, V.val, V.x, r);
    }
    if (!team_sync(t)) return false;
    const float* rp = V.rpre;
    amg_restrict(P, t, V, l, [=](int j) { return rp[j]; });
    return team_sync(t);
}

// Coarsest level: y = A_c^-1 b, one warp per row of the dense inverse.
__device__ __noinline__ bool ph_amg_dense(Ctx& C) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int n = P.nco, lane = threadIdx.x & 31;
    const int wpb = MM_BLOCK / 32;
    for (int row = t.rank * wpb + (int)(threadIdx.x >> 5); row < n; row += t.nb * wpb) {
        const float* a = P.ainv + (size_t)row * n;
        float s = 0.0f;
#pragma unroll 8
        for (int j = lane; j < n; j += 32) s += a[j] * P.bco[j];
        s = warp_sum_t<float>(s);
        if (lane == 0) P.yco[row] = s;
    }
    return team_sync(t);
}

// Up phase of level l: y = omega D^-1 (b + rpre) + U y_{l+1}.  At level 0,
// y is the preconditioned residual z; sums r.z and |r|^2.
__device__ __noinline__ bool ph_amg_up(Ctx& C, int l, double& rz, double& rr) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const Level& V = P.lev[l];
    const float* yc = (l + 1 == P.nlev) ? P.yco : P.lev[l + 1].y;
    const float* bv = (l == 0) ? P.pres32 : V.b;
    float acc[2] = {0.0f, 0.0f};
    // per row: b and omega D^-1 (b + rpre), loaded ahead of the product
    auto pre = [&](int r) {
        const float b = bv[r];
        return make_float2(b, V.omega * V.dinv[r] * (b + V.rpre[r]));
    };
    auto row = [&](int r, float s, float2 v) {
        const float y = v.y + s;
        V.y[r] = y;
        acc[0] += v.x * y;
        acc[1] += v.x * v.x;
    };
    if (l == 0) {
        level0_products(P, t, V.u_sptr, V.u_col, V.u_val, nullptr, yc, V.n, false, pre, row);
    } else {
        ROWS(r, V.n) {
            const float2 v = pre(r);
            row(r, sell_dot<16, float>(V.u_sptr, V.u_col, V.u_val, yc, r, 0), v);
        }
    }
    if (l > 0) return team_sync(t);
    double out[2];
    if (!team_sum_f32<2>(t, acc, out)) return false;
    rz = out[0];
    rr = out[1];
    return true;
}

// z = V-cycle(r) for r = pres32, whose smoothed iterate amg_x0 = omega
// D^-1 r has been written (and a barrier passed) by the caller.  Sums r.z,
// |r|^2.
__device__ bool amg_vcycle(Ctx& C, double& rz, double& rr) {
    const Problem& P = *C.P;
    for (int l = 0; l < P.nlev; ++l)
        if (!ph_amg_down(C, l)) return false;
    if (!ph_amg_dense(C)) return false;
    for (int l = P.nlev - 1; l >= 0; --l)
        if (!ph_amg_up(C, l, rz, rr)) return false;
    return true;
}

__device__ __forceinline__ bool use_amg(const Problem& P) { return P.prm.amg != 0 && P.nlev > 0; }

// r32 = r, z32 = M^-1 r32 (Jacobi or the V-cycle), delta = 0.  Sums: r.z, |r|^2.
__device__ bool ph_p32_init(Ctx& C, double& rz, double& rr) {
    const Problem& P = *C.P;
    Team& t = C.t;
    if (use_amg(P)) {
        ROWS(p, P.nphi) {
            const float r = (float)P.pres[p];
            P.pres32[p] = r;
            P.amg_x0[p] = P.amg_omega * P.dinvP32[p] * r;
            P.pdelta32[p] = 0.0f;
        }
        if (!team_sync(t)) return false;
        return amg_vcycle(C, rz, rr);
    }
    float acc[2] = {0.0f, 0.0f};
    double out[2];
    ROWS(p, P.nphi) {
        const float r = (float)P.pres[p];
        const float z = r * P.dinvP32[p];
        P.pres32[p] = r;
        P.pprec32[p] = z;
        P.pdelta32[p] = 0.0f;
        acc[0] += r * z;
        acc[1] += r * r;
    }
    if (!team_sum_f32<2>(t, acc, out)) return false;
    rz = out[0];
    rr = out[1];
    return true;
}

// FP32 direction step: d = z + beta d, q = K32 z + beta q.  Sum: d . q.
__device__ bool ph_p32_direction(Ctx& C, float beta, double& dq) {
    const Problem& P = *C.P;
    Team& t = C.t;
    float acc[1] = {0.0f};
    double out[1];
    const bool first = (beta == 0.0f);
    const float* z = P.pprec32;
    // per row: the new direction z + beta d and beta q, loaded ahead of the product
    auto pre = [&](int p) {
        return first ? make_float2(z[p], 0.0f) : make_float2(z[p] + beta * P.pdir32[p], beta * P.pq32[p]);
    };
    auto row = [&](int p, float s, float2 v) {
        const float qn = s + v.y;
        P.pdir32[p] = v.x;
        P.pq32[p] = qn;
        acc[0] += v.x * qn;
    };
    level0_products(P, t, P.k_sptr, P.k_col, P.Kp32, P.k_tab, z, P.nphi, true, pre, row);
    if (!team_sum_f32<1>(t, acc, out)) return false;
    dq = out[0];
    return true;
}

// delta += a d; r -= a q; z = M^-1 r.  Sums: r.z, |r|^2.
__device__ bool ph_p32_update(Ctx& C, float a, double& rz, double& rr) {
    const Problem& P = *C.P;
    Team& t = C.t;
    // Streaming pass in float4 (four rows per load; the FP32 vectors are
    // 256-byte aligned allocations), the n_phi % 4 tail in scalar form.
    // Measured on GB300 inside the solver kernel: 5.2 vs 8.1 us for a
    // three-vector pass over the bench mesh.
    const int n4 = P.nphi >> 2;
    float4* __restrict__ res4 = reinterpret_cast<float4*>(P.pres32);
    float4* __restrict__ del4 = reinterpret_cast<float4*>(P.pdelta32);
    const float4* __restrict__ dir4 = reinterpret_cast<const float4*>(P.pdir32);
    const float4* __restrict__ q4 = reinterpret_cast<const float4*>(P.pq32);
    const float4* __restrict__ dv4 = reinterpret_cast<const float4*>(P.dinvP32);
    if (use_amg(P)) {
        // no sums here: r.z and |r|^2 come with z from the V-cycle
        float4* __restrict__ x04 = reinterpret_cast<float4*>(P.amg_x0);
        const float om = P.amg_omega;
        ROWS(i, n4) {
            const float4 d = dir4[i], q = q4[i], r = res4[i], e = del4[i], w = dv4[i];
            const float4 nr = make_float4(r.x - a * q.x, r.y - a * q.y, r.z - a * q.z, r.w - a * q.w);
            del4[i] = make_float4(e.x + a * d.x, e.y + a * d.y, e.z + a * d.z, e.w + a * d.w);
            res4[i] = nr;
            x04[i] = make_float4(om * w.x * nr.x, om * w.y * nr.y, om * w.z * nr.z, om * w.w * nr.w);
        }
        ROWS(j, P.nphi - 4 * n4) {
            const int p = 4 * n4 + j;
            P.pdelta32[p] += a * P.pdir32[p];
            const float r = P.pres32[p] - a * P.pq32[p];
            P.pres32[p] = r;
            P.amg_x0[p] = om * P.dinvP32[p] * r;
        }
        if (!team_sync(t)) return false;
        return amg_vcycle(C, rz, rr);
    }
    float acc[2] = {0.0f, 0.0f};
    double out[2];
    float4* __restrict__ z4 = reinterpret_cast<float4*>(P.pprec32);
    ROWS(i, n4) {
        const float4 d = dir4[i], q = q4[i], r = res4[i], e = del4[i], w = dv4[i];
        const float4 nr = make_float4(r.x - a * q.x, r.y - a * q.y, r.z - a * q.z, r.w - a * q.w);
        const float4 z = make_float4(nr.x * w.x, nr.y * w.y, nr.z * w.z, nr.w * w.w);
        del4[i] = make_float4(e.x + a * d.x, e.y + a * d.y, e.z + a * d.z, e.w + a * d.w);
        res4[i] = nr;
        z4[i] = z;
        acc[0] += (nr.x * z.x + nr.y * z.y) + (nr.z * z.z + nr.w * z.w);
        acc[1] += (nr.x * nr.x + nr.y * nr.y) + (nr.z * nr.z + nr.w * nr.w);
    }
    ROWS(j, P.nphi - 4 * n4) {
        const int p = 4 * n4 + j;
        P.pdelta32[p] += a * P.pdir32[p];
        const float r = P.pres32[p] - a * P.pq32[p];
        const float z = r * P.dinvP32[p];
        P.pres32[p] = r;
        P.pprec32[p] = z;
        acc[0] += r * z;
        acc[1] += r * r;
    }
    if (!team_sum_f32<2>(t, acc, out)) return false;
    rz = out[0];
    rr = out[1];
    return true;
}

// FP64 refinement: phi += delta; r -= K delta (FP64 operator).  Sum: |r|^2.
__device__ bool ph_p64_refine(Ctx& C, double& rr) {
    const Problem& P = *C.P;
    Team& t = C.t;
    double acc[1] = {0.0};
    double dummy[1] = {0.0};
    const float* dl = P.pdelta32;
    ROWS(p, P.nphi) {
        const double s = sell_dot<8, double>(P.p_sptr, P.p_col, P.Kp, dl, p);
        P.phi[p] += (double)dl[p];
        const double r = P.pres[p] - s;
        P.pres[p] = r;
        acc[0] += r * r;
    }
    if (!team_reduce<1, 0>(t, acc, dummy)) return false;
    rr = acc[0];
    return true;
}

// Precision form of the potential solve: Algorithm 1 runs in FP32 on the
// correction equation K delta = r and keeps its direction across
// "reliable updates" (Clark et al., Comput. Phys. Commun. 181 (2010)):
// whenever the FP32 residual has dropped by inner_tol relative to its
// largest value since the last update (or below the target), the
// correction is folded into phi in FP64, the FP64 residual is recomputed
// from it (r -= K delta), and FP32 continues from that residual with the
// same direction.  Stops when the FP64 residual meets poisson_tol.
__device__ bool solve_potential_mixed(Ctx& C, double bb, double rr) {
    const Problem& P = *C.P;
    const double tol2 = C.ptol * C.ptol * bb;
    const double upd2 = P.prm.inner_tol * P.prm.inner_tol;
    if (rr < tol2) return true;
    double rz, r32;
    if (!ph_p32_init(C, rz, r32)) return false;
    double rmax = r32;
    float beta = 0.0f;
    long long k = 0;
    int updates = 0;
    while (k < P.prm.poisson_max_iter) {
        double dq;
        if (!ph_p32_direction(C, beta, dq)) return false;
        const float a = (float)(rz / dq);
        double rzn;
        if (!ph_p32_update(C, a, rzn, r32)) return false;
        ++k;
        if (r32 < upd2 * rmax || r32 < tol2) {
            // reliable update
            if (!ph_p64_refine(C, rr)) return false;
            C.mr++;
            ++updates;
            if (rr < tol2 || updates >= P.prm.max_refine) {
                C.mi += k + updates;
                return true;
            }
            if (!ph_p32_init(C, rzn, r32)) return false;
            rmax = r32;
        } else {
            rmax = fmax(rmax, r32);
        }
        beta = (float)(rzn / rz);
        rz = rzn;
    }
    // iteration cap: fold the pending correction into phi
    if (!ph_p64_refine(C, rr)) return false;
    C.mr++;
    C.mi += k + updates + 1;
    return true;
}

// Algorithm 1 on K_phi phi = D m (Sec. 3.1), warm-started from phi.
__device__ bool solve_potential(Ctx& C, int s) {
    const Problem& P = *C.P;
    double bb, rz, rr;
    if (!ph_pinit(C, s, bb, rz, rr)) return false;
    if (bb == 0.0) return ph_pzero(C);
    if (P.prm.precision == 1) return solve_potential_mixed(C, bb, rr);
    const double tol2 = C.ptol * C.ptol * bb;
    double beta = 0.0;
    long long k = 0;
    while (rr >= tol2 && k < P.prm.poisson_max_iter) {
        double pq;
        if (!ph_pdirection(C, P.pprec, beta, P.pdir[0], P.pq, pq)) return false;
        const double a = rz / pq;
        double rzn;
        if (!ph_pupdate(C, P.pdir[0], a, rzn, rr)) return false;
        beta = rzn / rz;
        rz = rzn;
        ++k;
    }
    C.mi += k;
    return true;
}

// Energy and gradient pass (Eq. energy, nablaLF, proj, opt2) at slot s:
// grad = C_A x + C_K x + D^T phi - w h; lambda = x . grad; g = grad - lambda x.
__device__ bool ph_gradient(Ctx& C, int s, bool trial) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    const double* x = P.X[s];
    double* gr = P.GR[s];
    double* gp = P.GP[s];
    double* lamv = P.LAM[s];
    const double h0 = C.h[0], h1 = C.h[1], h2 = C.h[2];
    // sums: exchange, anisotropy, Zeeman, phi.rhs, phi.r, dphi, M0, M1, M2, sum w
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double mx[1] = {0.0};
    ROWS(p, P.nphi) {
        acc[4] += P.phi[p] * P.pres[p];
        P.PHI[s][p] = P.phi[p];
        if (p < nm) {
            const int i = p;
            acc[3] += P.phi[i] * P.rhs[i];
            double c0, c1, c2, a0, a1, a2, t0, t1, t2;
            row_local(P, x, i, c0, c1, c2, a0, a1, a2);
            row_divT(P, P.phi, i, t0, t1, t2);
            const double x0 = x[i], x1 = x[nm + i], x2 = x[2 * nm + i];
            const double wi = P.w[i];
            const double g0 = 2.0 * c0 + a0 + t0 - wi * h0;
            const double g1 = 2.0 * c1 + a1 + t1 - wi * h1;
            const double g2 = 2.0 * c2 + a2 + t2 - wi * h2;
            acc[0] += x0 * c0 + x1 * c1 + x2 * c2;
            acc[1] += 0.5 * (x0 * a0 + x1 * a1 + x2 * a2);
            acc[2] -= wi * (h0 * x0 + h1 * x1 + h2 * x2);
            const double lam = x0 * g0 + x1 * g1 + x2 * g2;
            const double p0 = g0 - lam * x0, p1 = g1 - lam * x1, p2 = g2 - lam * x2;
            gr[i] = g0;
            gr[nm + i] = g1;
            gr[2 * nm + i] = g2;
            gp[i] = p0;
            gp[nm + i] = p1;
            gp[2 * nm + i] = p2;
            lamv[i] = lam;
            mx[0] = fmax(mx[0], fmax(fabs(p0), fmax(fabs(p1), fabs(p2))));
            if (trial)
                acc[5] += (p0 * P.d[i] + p1 * P.d[nm + i] + p2 * P.d[2 * nm + i]) / P.unorm[i];
            acc[6] += wi * x0;
            acc[7] += wi * x1;
            acc[8] += wi * x2;
            acc[9] += wi;
        }
    }
    if (!team_reduce<10, 1>(t, acc, mx)) return false;
    SlotScalars& S = C.sl[s];
    S.terms[0] = acc[0];
    S.terms[1] = acc[1];
    S.terms[2] = 0.5 * (acc[3] + acc[4]);   // phi.b - 1/2 phi.K phi, K phi = b - r
    S.terms[3] = acc[2];
    S.F = ((S.terms[0] + S.terms[1]) + S.terms[2]) + S.terms[3];
    S.dphi = acc[5];
    S.gmax = mx[0];
    S.M[0] = acc[6] / acc[9];
    S.M[1] = acc[7] / acc[9];
    S.M[2] = acc[8] / acc[9];
    return true;
}

// One function evaluation at slot s: at x_c + a d (trial) or at x_s as is.
// Warm start of a trial evaluation: phi is linear in m and the trial point
// is x_c + a d to first order, so phi(a) ~ PHI[c] + theta (PHI[ref] - PHI[c])
// with theta = a / a_ref (theta = 0: start from the current state's phi).
__device__ bool ph_phi_start(Ctx& C, int c, int ref, double theta) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const double* a = P.PHI[c];
    const double* b = P.PHI[ref];
    ROWS(p, P.nphi) P.phi[p] = (theta == 0.0) ? a[p] : a[p] + theta * (b[p] - a[p]);
    return team_sync(t);
}

__device__ bool ph_phi_restore(Ctx& C, int c) {
    const Problem& P = *C.P;
    Team& t = C.t;
    ROWS(p, P.nphi) P.phi[p] = P.PHI[c][p];
    return team_sync(t);
}

// One function evaluation at slot s: at x_c + a d (trial, potential warm
// start from the slots c and ref, see ph_phi_start) or at x_s as is (warm
// start from the last potential).
__device__ bool evaluate(Ctx& C, int c, int s, bool trial, double a, int ref = 0, double theta = 0.0) {
    if (trial && !ph_trial(C, c, s, a)) return false;
    if (trial && !ph_phi_start(C, c, ref, theta)) return false;
    if (!solve_potential(C, s)) return false;
    if (!ph_gradient(C, s, trial)) return false;
    C.evals++;
    return true;
}

// w = H(m) v (Eq. precond, magnetostatics dropped; last term only if
// keep_last_term).  With d given, the inner CG direction step follows by
// recurrence: d = ca v + beta d and hd = ca w + beta hd (= H d), in place,
// sum d . hd.  Without d, w is written to hd (sum v . w).
__device__ bool ph_hess(Ctx& C, int s, const double* v, double ca, double beta, double* d,
                        double* hd, double& dHd) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    const double* m = P.X[s];
    const double* lamv = P.LAM[s];
    const double* gr = P.GR[s];
    const bool keep = P.prm.keep_last_term != 0;
    const bool first = (beta == 0.0);
    double acc[1] = {0.0};
    double dummy[1] = {0.0};
    ROWS(i, nm) {
        double c0, c1, c2, k0, k1, k2;
        row_local(P, v, i, c0, c1, c2, k0, k1, k2);
        const double v0 = v[i], v1 = v[nm + i], v2 = v[2 * nm + i];
        const double Cv0 = 2.0 * c0 + k0;
        const double Cv1 = 2.0 * c1 + k1;
        const double Cv2 = 2.0 * c2 + k2;
        const double m0 = m[i], m1 = m[nm + i], m2 = m[2 * nm + i];
        const double mc = m0 * Cv0 + m1 * Cv1 + m2 * Cv2;
        const double lam = lamv[i];
        double w0 = Cv0 - mc * m0 - lam * v0;
        double w1 = Cv1 - mc * m1 - lam * v1;
        double w2 = Cv2 - mc * m2 - lam * v2;
        if (keep) {
            const double vg = v0 * gr[i] + v1 * gr[nm + i] + v2 * gr[2 * nm + i];
            w0 -= vg * m0;
            w1 -= vg * m1;
            w2 -= vg * m2;
        }
        if (d) {
            double dn[3] = {ca * v0, ca * v1, ca * v2};
            double hn[3] = {ca * w0, ca * w1, ca * w2};
            if (!first) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dn[c] += beta * d[c * nm + i];
                    hn[c] += beta * hd[c * nm + i];
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                d[c * nm + i] = dn[c];
                hd[c * nm + i] = hn[c];
                acc[0] += dn[c] * hn[c];
            }
        } else {
            hd[i] = w0;
            hd[nm + i] = w1;
            hd[2 * nm + i] = w2;
            acc[0] += v0 * w0 + v1 * w1 + v2 * w2;
        }
    }
    if (!team_reduce<1, 0>(t, acc, dummy)) return false;
    dHd = acc[0];
    return true;
}

// One application of an operator of Eq. (energy) (the operator entry
// point): MODE_DIV q = D v (v: idir[0], 3 x nm; q: pq, n_phi, zero on the
// air rows), MODE_DIVT w = D^T phi (phi: pdir[0]; w: ihd), MODE_LOCAL
// w = (C_A + C_K) v (v: idir[0]; w: ihd).
__device__ bool ph_operator(Ctx& C, int mode) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    if (mode == MODE_DIV) {
        ROWS(p, P.nphi) P.pq[p] = (p < nm) ? row_div(P, P.idir[0], p) : 0.0;
    } else if (mode == MODE_DIVT) {
        ROWS(i, nm) {
            double t0, t1, t2;
            row_divT(P, P.pdir[0], i, t0, t1, t2);
            P.ihd[i] = t0;
            P.ihd[nm + i] = t1;
            P.ihd[2 * nm + i] = t2;
        }
    } else {
        ROWS(i, nm) {
            double c0, c1, c2, a0, a1, a2;
            row_local(P, P.idir[0], i, c0, c1, c2, a0, a1, a2);
            P.ihd[i] = 2.0 * c0 + a0;
            P.ihd[nm + i] = 2.0 * c1 + a1;
            P.ihd[2 * nm + i] = 2.0 * c2 + a2;
        }
    }
    return team_sync(t);
}

// Algorithm 1 for H(m_s) y = g_s, y_0 = 0, Jacobi diag(C_A), exits li1-li3.
__device__ bool precond_solve(Ctx& C, int s) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    const int jmax = P.prm.jmax;
    if (jmax <= 0) {
        C.y_is_g = 1;
        return true;
    }
    const double* g = P.GP[s];
    // residual gr = H*0 + b with b = -g; preconditioned yv; direction -yv
    double acc[2] = {0.0, 0.0};
    double dummy[1] = {0.0};
    ROWS(i, nm) {
        const double di = P.dinvA[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double r = -g[c * nm + i];
            const double z = di * r;
            P.ires[c * nm + i] = r;
            P.iprec[c * nm + i] = z;
            P.isol[c * nm + i] = 0.0;
            acc[0] += r * z;
            acc[1] += r * r;
        }
    }
    if (!team_reduce<2, 0>(t, acc, dummy)) return false;
    double gy = acc[0];
    const double ng = sqrt(acc[1]);
    const double eps = fmin(0.5, sqrt(ng)) * ng;
    C.y_is_g = 0;
    if (ng < eps) return true;                  // y = 0 (only when g = 0 ... eps = 0)
    double beta = 0.0;
    int steps = 0;
    while (steps < jmax) {
        double dHd;
        // direction d = -yv + beta d and H d, by recurrence
        if (!ph_hess(C, s, P.iprec, -1.0, beta, P.idir[0], P.ihd, dHd)) return false;
        ++steps;
        C.li++;
        if (dHd <= 0.0) {                       // li2
            C.li2++;
            if (steps == 1) {
                C.y_is_g = 1;
                C.li2_first++;
            }
            return true;
        }
        const double a = gy / dHd;
        const double* dv = P.idir[0];
        double a2[2] = {0.0, 0.0};
        ROWS(i, nm) {
            const double di = P.dinvA[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int q = c * nm + i;
                P.isol[q] += a * dv[q];
                const double r = P.ires[q] + a * P.ihd[q];
                const double z = di * r;
                P.ires[q] = r;
                P.iprec[q] = z;
                a2[0] += r * z;
                a2[1] += r * r;
            }
        }
        if (!team_reduce<2, 0>(t, a2, dummy)) return false;
        if (sqrt(a2[1]) < eps) return true;     // li3
        beta = a2[0] / gy;
        gy = a2[0];
    }
    return true;                                // li1
}

// The precision form's preconditioner apply: precond_solve with H's
// products and the residual, preconditioned-residual, direction and
// H-direction vectors in FP32 (K_A, C_K and diag(C_A)^-1 as FP32 copies);
// m, lambda and the gradient are read from the FP64 state, the dots are
// FP32 products summed in FP64, the step length and beta stay FP64 scalars
// and the solution y accumulates in FP64 (the search direction is built from
// it).  The exits li1-li3 and their counters are those of precond_solve.
__device__ bool ph_hess32(Ctx& C, int s, const float* v, float beta, float* d, float* hd, double& dHd) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    const double* m = P.X[s];
    const double* lamv = P.LAM[s];
    const double* gr = P.GR[s];
    const bool keep = P.prm.keep_last_term != 0;
    const bool first = (beta == 0.0f);
    double acc[1] = {0.0};
    double dummy[1] = {0.0};
    ROWS(i, nm) {
        float c0, c1, c2;
        sell_dot3<8>(P.m_sptr, P.m_col, P.KA32, v, nm, i, c0, c1, c2);
        const float v0 = v[i], v1 = v[nm + i], v2 = v[2 * nm + i];
        const float kxx = P.CK32[i], kxy = P.CK32[nm + i], kxz = P.CK32[2 * nm + i];
        const float kyy = P.CK32[3 * nm + i], kyz = P.CK32[4 * nm + i], kzz = P.CK32[5 * nm + i];
        const float Cv0 = 2.0f * c0 + (kxx * v0 + kxy * v1 + kxz * v2);
        const float Cv1 = 2.0f * c1 + (kxy * v0 + kyy * v1 + kyz * v2);
        const float Cv2 = 2.0f * c2 + (kxz * v0 + kyz * v1 + kzz * v2);
        const float m0 = (float)m[i], m1 = (float)m[nm + i], m2 = (float)m[2 * nm + i];
        const float mc = m0 * Cv0 + m1 * Cv1 + m2 * Cv2;
        const float lam = (float)lamv[i];
        float w[3] = {Cv0 - mc * m0 - lam * v0, Cv1 - mc * m1 - lam * v1, Cv2 - mc * m2 - lam * v2};
        if (keep) {
            const float vg = v0 * (float)gr[i] + v1 * (float)gr[nm + i] + v2 * (float)gr[2 * nm + i];
            w[0] -= vg * m0;
            w[1] -= vg * m1;
            w[2] -= vg * m2;
        }
        const float vv[3] = {v0, v1, v2};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // d = -v + beta d, hd = -H v + beta hd (= H d)
            float dn = -vv[c], hn = -w[c];
            if (!first) {
                dn += beta * d[c * nm + i];
                hn += beta * hd[c * nm + i];
            }
            d[c * nm + i] = dn;
            hd[c * nm + i] = hn;
            acc[0] += (double)(dn * hn);
        }
    }
    if (!team_reduce<1, 0>(t, acc, dummy)) return false;
    dHd = acc[0];
    return true;
}

__device__ bool precond_solve32(Ctx& C, int s) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    const int jmax = P.prm.jmax;
    if (jmax <= 0) {
        C.y_is_g = 1;
        return true;
    }
    const double* g = P.GP[s];
    double acc[2] = {0.0, 0.0};
    double dummy[1] = {0.0};
    ROWS(i, nm) {
        const float di = P.dinvA32[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float r = (float)(-g[c * nm + i]);
            const float z = di * r;
            P.ires32[c * nm + i] = r;
            P.iprec32[c * nm + i] = z;
            P.isol[c * nm + i] = 0.0;
            acc[0] += (double)(r * z);
            acc[1] += (double)(r * r);
        }
    }
    if (!team_reduce<2, 0>(t, acc, dummy)) return false;
    double gy = acc[0];
    const double ng = sqrt(acc[1]);
    const double eps = fmin(0.5, sqrt(ng)) * ng;
    C.y_is_g = 0;
    if (ng < eps) return true;
    double beta = 0.0;
    int steps = 0;
    while (steps < jmax) {
        double dHd;
        if (!ph_hess32(C, s, P.iprec32, (float)beta, P.idir32, P.ihd32, dHd)) return false;
        ++steps;
        C.li++;
        if (dHd <= 0.0) {                       // li2
            C.li2++;
            if (steps == 1) {
                C.y_is_g = 1;
                C.li2_first++;
            }
            return true;
        }
        const double a = gy / dHd;
        const float af = (float)a;
        double a2[2] = {0.0, 0.0};
        ROWS(i, nm) {
            const float di = P.dinvA32[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int q = c * nm + i;
                P.isol[q] += a * (double)P.idir32[q];
                const float r = P.ires32[q] + af * P.ihd32[q];
                const float z = di * r;
                P.ires32[q] = r;
                P.iprec32[q] = z;
                a2[0] += (double)(r * z);
                a2[1] += (double)(r * r);
            }
        }
        if (!team_reduce<2, 0>(t, a2, dummy)) return false;
        if (sqrt(a2[1]) < eps) return true;     // li3
        beta = a2[0] / gy;
        gy = a2[0];
    }
    return true;                                // li1
}

// The preconditioner apply of the configured form.
__device__ bool precond_apply(Ctx& C, int s) {
    return C.P->prm.precision ? precond_solve32(C, s) : precond_solve(C, s);
}

// beta*ZA dots between slot a (new gradient gn) and slot c (old gradient go)
// with y the preconditioned gn and d the previous direction:
//   y.gn, y.go, (gn-go).y, (gn-go).d, gn.d, gn.gn, gn.go, (gn-go).gn
__device__ bool ph_dir_dots(Ctx& C, int a, int c, double (&dots)[8]) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    const double* y = C.y_is_g ? P.GP[a] : P.isol;
    const double* gn = P.GP[a];
    const double* go = P.GP[c];
    double dummy[1] = {0.0};
    for (int k = 0; k < 8; ++k) dots[k] = 0.0;
    ROWS(i, nm) {
#pragma unroll
        for (int q3 = 0; q3 < 3; ++q3) {
            const int q = q3 * nm + i;
            const double yy = y[q], n = gn[q], o = go[q], dd = P.d[q];
            const double dg = n - o;
            dots[0] += yy * n;
            dots[1] += yy * o;
            dots[2] += dg * yy;
            dots[3] += dg * dd;
            dots[4] += n * dd;
            dots[5] += n * n;
            dots[6] += n * o;
            dots[7] += dg * n;
        }
    }
    return team_reduce<8, 0>(t, dots, dummy);
}

// d = -v + beta d (kind 1: v = y; kind 2: v = g; kind 3: d = -g), max_i |d_i|.
__device__ bool ph_dir_write(Ctx& C, int a, int kind, double beta, double& dmax) {
    const Problem& P = *C.P;
    Team& t = C.t;
    const int nm = P.nm;
    const double* y = C.y_is_g ? P.GP[a] : P.isol;
    const double* v = (kind == 1) ? y : P.GP[a];
    const double b = (kind == 3) ? 0.0 : beta;   // b == 0: d_old is not read
    double mx[1] = {0.0};
    double dummy[1] = {0.0};
    ROWS(i, nm) {
        double n2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int q = c * nm + i;
            const double dn = (b == 0.0) ? -v[q] : -v[q] + b * P.d[q];
            P.d[q] = dn;
            n2 += dn * dn;
        }
        mx[0] = fmax(mx[0], sqrt(n2));
    }
    if (!team_reduce<0, 1>(t, dummy, mx)) return false;
    dmax = mx[0];
    return true;
}

__device__ __forceinline__ double beta_za(double y_gn, double y_go, double dg_y, double dg_d) {
    if (y_gn > y_go) return (dg_d == 0.0) ? 0.0 : dg_y / dg_d;
    return 0.0;
}

// The direction update of Algorithm 3/4 with y the preconditioned new
// gradient: beta*ZA (restarted Hestenes-Stiefel), beta*FR = g+.y+ / g.y
// (Eq. FRstar), beta*PRP = (g+ - g).y+ / g.y (Eq. PRPstar), g.y = gy_prev
// of the last direction (0 gives beta = 0).
__device__ __forceinline__ double beta_rule(int rule, double y_gn, double y_go, double dg_y, double dg_d,
                                            double gy_prev) {
    if (rule == 1) return (gy_prev == 0.0) ? 0.0 : y_gn / gy_prev;
    if (rule == 2) return (gy_prev == 0.0) ? 0.0 : dg_y / gy_prev;
    return beta_za(y_gn, y_go, dg_y, dg_d);
}

// New direction with beta*ZA and the descent safeguard; returns g.d.
__device__ bool direction(Ctx& C, int a, int c, bool initial, double& dmax, double& gd) {
    double dots[8];
    if (!ph_dir_dots(C, a, c, dots)) return false;
    const double y_gn = dots[0], y_go = dots[1], dg_y = dots[2], dg_d = dots[3];
    const double gn_d = dots[4], gn_gn = dots[5], gn_go = dots[6], dg_gn = dots[7];
    const int rule = C.P->prm.beta_rule;
    int kind = 1;
    double beta = 0.0;
    if (initial) {
        gd = -y_gn;
        if (gd >= 0.0) {
            kind = 3;
            gd = -gn_gn;
            C.steepest++;
        }
    } else {
        beta = beta_rule(rule, y_gn, y_go, dg_y, dg_d, C.gy_prev);
        gd = -y_gn + beta * gn_d;
        if (gd >= 0.0) {
            beta = beta_rule(rule, gn_gn, gn_go, dg_gn, dg_d, C.gy_prev);
            kind = 2;
            gd = -gn_gn + beta * gn_d;
            C.restarts++;
            if (gd >= 0.0) {
                kind = 3;
                beta = 0.0;
                gd = -gn_gn;
                C.steepest++;
            }
        }
    }
    C.gy_prev = (kind == 1) ? y_gn : gn_gn;     // g.y of the direction built (y = g after the safeguard)
    return ph_dir_write(C, a, kind, beta, dmax);
}

__device__ __forceinline__ bool cubic_step(double f0, double g0, double a, double f1, double g1,
                                           double& out) {
    const double d1 = g0 + g1 - 3.0 * (f1 - f0) / a;
    const double disc = d1 * d1 - g0 * g1;
    if (!(disc > 0.0)) return false;
    const double d2 = sqrt(disc);
    const double den = g1 - g0 + 2.0 * d2;
    if (den == 0.0) return false;
    out = a - a * (g1 + d2 - d1) / den;
    return isfinite(out);
}

// Algorithm 4 at the current field from slot C.cur.
__device__ int minimize(Ctx& C, int& cur) {
    const Problem& P = *C.P;
    const Params& prm = P.prm;
    int c = cur;
    if (!evaluate(C, c, c, false, 0.0)) return ST_TIMEOUT;
    if (!precond_apply(C, c)) return ST_TIMEOUT;
    double dmax, gd;
    if (!direction(C, c, c, true, dmax, gd)) return ST_TIMEOUT;
    double a_prev = 1.0;
    int status = ST_RUNNING;
    if (!isfinite(C.sl[c].F)) status = ST_NONFINITE;
    else if (C.sl[c].gmax == 0.0) status = ST_OK;
    const double sq_tau = sqrt(prm.tau_F);
    const double cb_tau = cbrt(prm.tau_F);
    double dF_prev = -1.0;                      // last accepted decrease (none yet)
    while (status == ST_RUNNING && C.nli < prm.max_iter) {
        const double F0 = C.sl[c].F;
        // potential tolerance of this iteration's evaluations (poisson_sched):
        // loosened while the last decrease is far above the t1 threshold, so
        // that the energy error (quadratic in the potential error) stays far
        // below the decrease the line search resolves
        C.ptol = prm.poisson_tol;
        if (prm.poisson_sched && dF_prev > 0.0) {
            const double q = dF_prev / (prm.tau_F * (1.0 + fabs(F0)));
            if (q > 100.0) C.ptol = fmin(prm.poisson_tol_max, fmax(prm.poisson_tol, prm.poisson_tol * sqrt(q) / 10.0));
        }
        const double dphi0 = gd;
        const double a_max = prm.theta_max / dmax;
        const double a_t = fmin(a_prev, a_max);
        const int ts = (c + 1) % MM_NSLOT, ss = (c + 2) % MM_NSLOT;
        if (!evaluate(C, c, ts, true, a_t, c, 0.0)) return ST_TIMEOUT;
        double a_s;
        if (!cubic_step(F0, dphi0, a_t, C.sl[ts].F, C.sl[ts].dphi, a_s))
            a_s = (C.sl[ts].dphi < 0.0) ? 4.0 * a_t : 0.5 * a_t;
        a_s = fmin(fmax(a_s, 0.1 * a_t), fmin(4.0 * a_t, a_max));
        if (!evaluate(C, c, ss, true, a_s, ts, a_s / a_t)) return ST_TIMEOUT;
        int b;
        double a_b;
        if (C.sl[ss].F <= C.sl[ts].F) {
            b = ss;
            a_b = a_s;
        } else {
            b = ts;
            a_b = a_t;
        }
        if (!(C.sl[b].F <= F0 + prm.c1 * a_b * dphi0)) {
            bool found = false;
            double a = 0.5 * fmin(a_t, a_s);
            for (int k = 0; k < prm.max_backtrack; ++k) {
                if (!evaluate(C, c, ts, true, a, ss, a / a_s)) return ST_TIMEOUT;
                C.ls_extra++;
                if (C.sl[ts].F <= F0 + prm.c1 * a * dphi0) {
                    b = ts;
                    a_b = a;
                    found = true;
                    break;
                }
                a *= 0.5;
            }
            if (!found) {
                status = ST_STALLED;
                break;
            }
        }
        C.nli++;
        const SlotScalars& S = C.sl[b];
        dF_prev = F0 - S.F;
        if (!isfinite(S.F)) {
            status = ST_NONFINITE;
            break;
        }
        const bool t1 = F0 - S.F < prm.tau_F * (1.0 + fabs(S.F));
        const bool t2 = S.xdiff < sq_tau * (1.0 + S.xmax);
        const bool t3 = S.gmax < cb_tau * (1.0 + fabs(S.F));
        if (!precond_apply(C, b)) return ST_TIMEOUT;
        if (!direction(C, b, c, false, dmax, gd)) return ST_TIMEOUT;
        c = b;
        a_prev = a_b;
        if (t1 && t2 && t3) status = ST_OK;
    }
    if (status == ST_RUNNING) status = ST_NOT_CONVERGED;
    // leave the accepted state's potential as the working one (the next
    // field step starts from it; the host reads it)
    if (!ph_phi_restore(C, c)) return ST_TIMEOUT;
    cur = c;
    return status;
}

}  // namespace

// The solver on one team of nb blocks (this block is number rank).
__device__ __forceinline__ void solver_body(const Problem& P, int nb, int rank) {
    Ctx C;
    C.P = &P;
    C.t.nb = nb;
    C.t.rank = rank;
    C.t.count = reinterpret_cast<unsigned long long*>(P.bar);
    C.t.err = P.err;
    C.t.part = P.partials;
    C.t.epoch = 0;
    C.t.dead = false;
    C.evals = C.nli = C.li = C.mi = C.ls_extra = C.mr = 0;
    C.li2 = C.li2_first = C.restarts = C.steepest = 0;
    C.y_is_g = 0;
    C.ptol = P.prm.poisson_tol;
    C.gy_prev = 0.0;
    int cur = P.state->cur;
    C.h[0] = P.state->h[0];
    C.h[1] = P.state->h[1];
    C.h[2] = P.state->h[2];
    int status = ST_OK;
    switch (P.mode) {
        case MODE_MINIMIZE:
            status = minimize(C, cur);
            break;
        case MODE_EVAL:
            if (!evaluate(C, cur, cur, false, 0.0)) status = ST_TIMEOUT;
            break;
        case MODE_PRECOND:
            if (!precond_apply(C, cur)) status = ST_TIMEOUT;
            break;
        case MODE_HESS: {
            // input v in idir[0], output in ihd
            double vHv;
            if (!ph_hess(C, cur, P.idir[0], 1.0, 0.0, nullptr, P.ihd, vHv)) status = ST_TIMEOUT;
            break;
        }
        case MODE_KPHI: {
            // input in pdir[0], output in pq
            if (!ph_pmatvec(C, P.pdir[0], P.pq)) status = ST_TIMEOUT;
            break;
        }
        case MODE_DIV:
        case MODE_DIVT:
        case MODE_LOCAL:
            if (!ph_operator(C, P.mode)) status = ST_TIMEOUT;
            break;
        default:
            status = ST_TIMEOUT;
    }
    if (C.t.dead) status = ST_TIMEOUT;
    if (rank == 0 && threadIdx.x == 0) {
        DevState* st = P.state;
        st->cur = cur;
        st->status = status;
        st->evals = C.evals;
        st->nli = C.nli;
        st->li = C.li;
        st->mi = C.mi;
        st->ls_extra = C.ls_extra;
        st->mr = C.mr;
        st->li2 = C.li2;
        st->li2_first = C.li2_first;
        st->restarts = C.restarts;
        st->steepest = C.steepest;
        if (P.mode == MODE_MINIMIZE || P.mode == MODE_EVAL) {
            const SlotScalars& S = C.sl[cur];
            st->F = S.F;
            for (int k = 0; k < 4; ++k) st->terms[k] = S.terms[k];
            for (int k = 0; k < 3; ++k) st->M[k] = S.M[k];
            st->gmax = S.gmax;
        }
        st->y_is_g = C.y_is_g;
    }
}

// One instantiation per occupancy target (minimum resident blocks per SM),
// each compiled in its own translation unit (mm_kern_*.cu); the host picks
// one through solver_kernel() / solver_batch_kernel().
template <int MINB>
__global__ void __launch_bounds__(MM_BLOCK, MINB) k_solver(const __grid_constant__ Problem P) {
    solver_body(P, (int)gridDim.x, (int)blockIdx.x);
}

// Batched form: the grid is split into teams, team j = blocks
// [team_first[j], team_first[j+1]) runs the solver on problem j.  Teams only
// synchronise internally, so problems of different sizes and iteration
// counts proceed independently inside one launch.
template <int MINB>
__global__ void __launch_bounds__(MM_BLOCK, MINB) k_solver_batch(const Problem* __restrict__ probs,
                                                                  const int* __restrict__ team_first, int nteams) {
    int lo = 0, hi = nteams;                 // team_first[lo] <= blockIdx.x < team_first[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (team_first[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid;
    }
    const int first = team_first[lo];
    solver_body(probs[lo], team_first[lo + 1] - first, (int)blockIdx.x - first);
}

}  // namespace mm
