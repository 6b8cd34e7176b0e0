// Energy and gradient with no device allocation in the call.
//
// Some callers cannot call cudaMalloc (or let a library do it for them): a
// process whose device memory is handed in full to its own pool allocator
// or held to a fixed quota, or a latency-bound loop that cannot afford the
// device-wide synchronisation that cudaFree implies.  For them
// mm_energy_gradient_noalloc evaluates the potential solve and the energy /
// gradient pass of the solver kernel (the MODE_EVAL path of k_solver) with
// every work vector, reduction partial and barrier word placed in one
// file-scope device array of fixed size instead of context buffers.  The
// operators assembled by mm_upload_mesh are read, never written.
//
// The array is held by every GPU that loads the library until the process
// exits.  Every call shares it and it keeps the last call's contents; the
// call clears what must start at zero (barrier words, error flag, the
// potential's starting guess).  Calls that overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mmncg.h"
#include "mm_internal.cuh"

namespace {

constexpr size_t kScratchDoubles = (size_t)1 << 20;   // 8 MiB
constexpr double kMu0 = 4e-7 * 3.14159265358979323846;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;

// Device address of the scratch array on the current device, looked up on
// every call with that device current (a cheap host call; a cached address
// would go stale if the caller reset the device and made a new context).
int scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return MM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return MM_ERR_CUDA;
    }
    *out = (double*)p;
    return MM_OK;
}

inline size_t up32(size_t n) { return (n + 31) & ~(size_t)31; }   // 256-byte granules

__global__ void k_noalloc_prep(int nm, const int* mag_nodes, const double* m_nodes, double* X,
                               mm::DevState* st, double h0, double h1, double h2, int* bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        memset(st, 0, sizeof(mm::DevState));
        st->cur = 0;
        st->h[0] = h0;
        st->h[1] = h1;
        st->h[2] = h2;
    }
    if (i >= nm) return;
    const long long n = mag_nodes[i];
    const double a = m_nodes[3 * n], b = m_nodes[3 * n + 1], c = m_nodes[3 * n + 2];
    const double r = sqrt(a * a + b * b + c * c);
    const bool ok = (r > 0.0) && isfinite(r);
    X[i] = ok ? a / r : 0.0;
    X[nm + i] = ok ? b / r : 0.0;
    X[2 * nm + i] = ok ? c / r : 1.0;
    if (!ok) atomicExch(bad, 1);
}

__global__ void k_noalloc_out(int nm, const int* mag_nodes, const double* g, double* grad_nodes,
                              const mm::DevState* st, double EJ, double* energy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && energy) {
        energy[0] = st->F * EJ;
        for (int k = 0; k < 4; ++k) energy[1 + k] = st->terms[k] * EJ;
    }
    if (i >= nm || !grad_nodes) return;
    const long long n = mag_nodes[i];
    grad_nodes[3 * n] = g[i];
    grad_nodes[3 * n + 1] = g[nm + i];
    grad_nodes[3 * n + 2] = g[2 * nm + i];
}

}  // namespace

extern "C" int mm_energy_gradient_noalloc(mm_ctx* ctx, const double* m_dev, const mm_params* p,
                                          double* grad_dev, int projected, double* energy_dev) {
    mm::CtxView v;
    if (!ctx || mm::ctx_view(ctx, &v) != MM_OK) return MM_ERR_ARG;
    if (!v.has_mesh) return mm::ctx_fail(ctx, MM_ERR_STATE, "no mesh uploaded");
    if (!m_dev || !energy_dev) return mm::ctx_fail(ctx, MM_ERR_ARG, "m_dev and energy_dev are required");
    mm_params d;
    mm_default_params(&d);
    if (!p) p = &d;
    if (!(p->poisson_tol > 0.0) || p->poisson_max_iter < 1)
        return mm::ctx_fail(ctx, MM_ERR_ARG, "poisson_tol must be > 0 and poisson_max_iter >= 1");
    if (cudaSetDevice(v.device) != cudaSuccess) return mm::ctx_fail(ctx, MM_ERR_CUDA, "cudaSetDevice failed");

    // layout of the scratch array (doubles, 256-byte aligned pieces)
    const size_t nm = (size_t)v.nm, np = (size_t)v.nphi;
    size_t off = 0;
    auto take = [&](size_t n) {
        const size_t o = off;
        off += up32(n);
        return o;
    };
    const size_t o_state = take((sizeof(mm::DevState) + 7) / 8);
    const size_t o_bar = take(32);                  // 64 unsigned
    const size_t o_err = take(1);
    const size_t o_bad = take(1);
    const size_t o_part = take(2 * (size_t)MM_MAXRED * v.blocks);
    const size_t o_X = take(3 * nm), o_GR = take(3 * nm), o_GP = take(3 * nm);
    const size_t o_LAM = take(nm), o_un = take(nm), o_rhs = take(nm);
    const size_t o_phi = take(np), o_res = take(np), o_prec = take(np);
    const size_t o_d0 = take(np), o_d1 = take(np), o_q = take(np);
    if (off > kScratchDoubles) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "problem needs %.2f MiB of scratch; the no-allocation entry point holds %.0f MiB "
                 "(11 n_mag + 6 n_phi doubles plus reduction space)",
                 off * 8.0 / (1 << 20), kScratchDoubles * 8.0 / (1 << 20));
        return mm::ctx_fail(ctx, MM_ERR_ARG, msg);
    }
    double* S = nullptr;
    if (scratch_address(v.device, &S) != MM_OK)
        return mm::ctx_fail(ctx, MM_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");

    cudaStream_t st = (cudaStream_t)v.stream;
    mm::Problem Q = *v.P;                           // operators: read only
    mm::DevState* dstate = (mm::DevState*)(S + o_state);
    double* X = S + o_X;
    for (int s = 0; s < MM_NSLOT; ++s) {
        Q.X[s] = X;
        Q.GR[s] = S + o_GR;
        Q.GP[s] = S + o_GP;
        Q.LAM[s] = S + o_LAM;
    }
    Q.unorm = S + o_un;
    Q.d = S + o_un;                                  // not read by an evaluation
    Q.isol = Q.ires = Q.iprec = Q.ihd = S + o_GP;    // not used by an evaluation
    Q.idir[0] = Q.idir[1] = S + o_GP;
    Q.phi = S + o_phi;
    for (int s = 0; s < MM_NSLOT; ++s) Q.PHI[s] = S + o_phi;   // an evaluation saves phi in place
    Q.rhs = S + o_rhs;
    Q.pres = S + o_res;
    Q.pprec = S + o_prec;
    Q.pdir[0] = S + o_d0;
    Q.pdir[1] = S + o_d1;
    Q.pq = S + o_q;
    Q.partials = S + o_part;
    Q.bar = (unsigned*)(S + o_bar);
    Q.err = (int*)(S + o_err);
    Q.state = dstate;
    Q.mode = mm::MODE_EVAL;
    Q.prm.tau_F = p->tau_F;
    Q.prm.jmax = p->jmax;
    Q.prm.max_iter = p->max_iter;
    Q.prm.theta_max = p->theta_max;
    Q.prm.c1 = p->c1;
    Q.prm.max_backtrack = p->max_backtrack;
    Q.prm.keep_last_term = p->keep_last_term;
    Q.prm.poisson_tol = p->poisson_tol;
    Q.prm.poisson_max_iter = p->poisson_max_iter;
    Q.prm.precision = 0;                            // the FP64 evaluation only
    Q.prm.inner_tol = p->inner_tol;
    Q.prm.max_refine = p->max_refine;
    Q.prm.amg = 0;
    Q.prm.beta_rule = 0;
    Q.prm.poisson_sched = 0;
    Q.prm.poisson_tol_max = p->poisson_tol;
    Q.nlev = 0;
    Q.pres32 = Q.pprec32 = Q.pdir32 = Q.pq32 = Q.pdelta32 = nullptr;

    const double hs = 1.0 / (kMu0 * v.Mref);
    int* bad = (int*)(S + o_bad);
    cudaError_t e;
    // clear what must start at zero: barrier words, error flag, the flag of
    // bad input vectors (cleared on the stream before the kernel that sets
    // it: blocks of one launch run in no fixed order), potential
    if ((e = cudaMemsetAsync(Q.bar, 0, 64 * sizeof(unsigned), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(Q.err, 0, sizeof(int), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(bad, 0, sizeof(int), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(Q.phi, 0, np * sizeof(double), st)) != cudaSuccess)
        return mm::ctx_fail(ctx, MM_ERR_CUDA, cudaGetErrorString(e));
    const int nb = (int)((nm + 255) / 256);
    k_noalloc_prep<<<nb > 0 ? nb : 1, 256, 0, st>>>(v.nm, v.mag_nodes, m_dev, X, dstate, v.field_T[0] * hs,
                                                   v.field_T[1] * hs, v.field_T[2] * hs, bad);
    if ((e = cudaGetLastError()) != cudaSuccess) return mm::ctx_fail(ctx, MM_ERR_CUDA, cudaGetErrorString(e));
    void* args[] = {(void*)&Q};
    if ((e = cudaLaunchCooperativeKernel(v.kernel, dim3(v.blocks), dim3(MM_BLOCK), args, 0, st)) != cudaSuccess)
        return mm::ctx_fail(ctx, MM_ERR_CUDA, cudaGetErrorString(e));
    if (grad_dev &&
        (e = cudaMemsetAsync(grad_dev, 0, (size_t)v.n_nodes * 3 * sizeof(double), st)) != cudaSuccess)
        return mm::ctx_fail(ctx, MM_ERR_CUDA, cudaGetErrorString(e));
    const double EJ = kMu0 * v.Mref * v.Mref * 1e-27;
    k_noalloc_out<<<nb > 0 ? nb : 1, 256, 0, st>>>(v.nm, v.mag_nodes, projected ? Q.GP[0] : Q.GR[0], grad_dev,
                                                  dstate, EJ, energy_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return mm::ctx_fail(ctx, MM_ERR_CUDA, cudaGetErrorString(e));
    int flags[2] = {0, 0};
    mm::DevState hs_state;
    if ((e = cudaMemcpyAsync(&flags[0], Q.err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&flags[1], bad, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&hs_state, dstate, sizeof(mm::DevState), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return mm::ctx_fail(ctx, MM_ERR_CUDA, cudaGetErrorString(e));
    if (flags[1]) return mm::ctx_fail(ctx, MM_ERR_NONFINITE, "magnetisation has a zero or non-finite vector");
    if (flags[0] || hs_state.status == mm::ST_TIMEOUT)
        return mm::ctx_fail(ctx, MM_ERR_DEVICE_TIMEOUT, "a device barrier wait ran out");
    if (!std::isfinite(hs_state.F)) return mm::ctx_fail(ctx, MM_ERR_NONFINITE, "non-finite energy");
    return MM_OK;
}
