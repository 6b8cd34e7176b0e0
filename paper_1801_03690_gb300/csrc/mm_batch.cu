// Batched minimisation: many independent problems (contexts on one device)
// in one persistent cooperative launch, each problem on its own team of
// blocks (k_solver_batch), the field loop replayed from a captured CUDA
// graph, and an autotuner for the kernel instantiation and the team split.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mmncg.h"
#include "mm_internal.cuh"

namespace {

constexpr double kMu0 = 4e-7 * 3.14159265358979323846;
constexpr int kBarWords = 64;      // per team: [0..1] the 64-bit arrival counter
constexpr int kErrWords = 32;      // per team error flag, one 128-byte line

__global__ void k_batch_fields(int n, const double* fields, const int* step, mm::DevState* const* states) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double* f = fields + ((size_t)(*step) * n + t) * 3;
    states[t]->h[0] = f[0];
    states[t]->h[1] = f[1];
    states[t]->h[2] = f[2];
}

__global__ void k_batch_record(int n, mm::DevState* const* states, mm::DevState* hist, int* step) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) hist[(size_t)(*step) * n + t] = *states[t];
    __syncthreads();
    if (t == 0) *step += 1;
}

__global__ void k_batch_status(int n, mm::DevState* const* states, mm::DevState* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = *states[t];
}

}  // namespace

struct mm_batch {
    int n = 0;
    int device = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    std::vector<mm_ctx*> ctxs;
    std::vector<mm::CtxView> views;
    std::vector<int64_t> work;
    int variant = 3;
    double gamma = 1.0;
    int tile_rows = 0, restrict_lanes = 0;   // tile shape of every member (0 = default)
    int blocks = 0;
    std::vector<int> team_first;
    std::string err;
    // device
    mm::Problem* d_probs = nullptr;
    int* d_team_first = nullptr;
    double* d_part = nullptr;
    size_t part_cap = 0;
    unsigned* d_bar = nullptr;
    int* d_err = nullptr;
    mm::DevState** d_states = nullptr;
    mm::DevState* d_stat = nullptr;
    mm::DevState* h_stat = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

int bfail(mm_batch* b, int code, const char* msg) {
    if (b) b->err = msg;
    return code;
}

#define BK(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return bfail(b, MM_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

mm::Params conv(const mm_params* p) {
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
    q.inner_tol = p->inner_tol;
    q.max_refine = p->max_refine;
    q.amg = p->amg;
    q.beta_rule = p->beta_rule;
    q.poisson_sched = p->poisson_sched;
    q.poisson_tol_max = p->poisson_tol_max;
    return q;
}

// Plan the grid for the current variant/gamma and upload the per-team
// problem descriptors.
int prepare(mm_batch* b, const mm::Params& prm) {
    BK(cudaSetDevice(b->device));
    for (int t = 0; t < b->n; ++t)      // members may have been re-uploaded
        if (mm::ctx_view(b->ctxs[t], &b->views[t]) != MM_OK || !b->views[t].has_mesh)
            return bfail(b, MM_ERR_STATE, "a member context has no mesh");
    const void* kern = mm::solver_batch_kernel(b->variant);
    int bps = 0;
    BK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, MM_BLOCK, 0));
    bps = std::min(bps, b->variant);
    if (bps < 1) return bfail(b, MM_ERR_CUDA, "batched solver kernel does not fit on an SM");
    const int total = bps * b->nsm;
    if (b->n > total) return bfail(b, MM_ERR_ARG, "more problems than co-resident blocks in one launch");
    std::vector<int32_t> tb(b->n);
    int rc = mm_batch_plan(b->n, b->work.data(), total, b->gamma, tb.data());
    if (rc) return bfail(b, rc, "team planning failed");
    b->blocks = total;
    b->team_first.assign(b->n + 1, 0);
    for (int t = 0; t < b->n; ++t) b->team_first[t + 1] = b->team_first[t] + tb[t];
    const size_t need = 2 * (size_t)MM_MAXRED * total;
    if (need > b->part_cap) {
        if (b->d_part) cudaFree(b->d_part);
        b->d_part = nullptr;
        BK(cudaMalloc(&b->d_part, need * sizeof(double)));
        b->part_cap = need;
    }
    std::vector<mm::Problem> probs(b->n);
    for (int t = 0; t < b->n; ++t) {
        mm::Problem q = *b->views[t].P;
        q.prm = prm;
        q.mode = mm::MODE_MINIMIZE;
        q.tile_rows = b->tile_rows;
        q.restrict_lanes = b->restrict_lanes;
        q.partials = b->d_part + 2 * (size_t)MM_MAXRED * b->team_first[t];
        q.bar = b->d_bar + (size_t)kBarWords * t;
        q.err = b->d_err + (size_t)kErrWords * t;
        probs[t] = q;
    }
    BK(cudaMemcpy(b->d_probs, probs.data(), b->n * sizeof(mm::Problem), cudaMemcpyHostToDevice));
    BK(cudaMemcpy(b->d_team_first, b->team_first.data(), (b->n + 1) * sizeof(int), cudaMemcpyHostToDevice));
    return MM_OK;
}

int enqueue_launch(mm_batch* b) {
    BK(cudaMemsetAsync(b->d_bar, 0, (size_t)kBarWords * b->n * sizeof(unsigned), b->stream));
    BK(cudaMemsetAsync(b->d_err, 0, (size_t)kErrWords * b->n * sizeof(int), b->stream));
    const mm::Problem* probs = b->d_probs;
    const int* tf = b->d_team_first;
    int n = b->n;
    void* args[] = {(void*)&probs, (void*)&tf, (void*)&n};
    BK(cudaLaunchCooperativeKernel(mm::solver_batch_kernel(b->variant), dim3(b->blocks), dim3(MM_BLOCK), args, 0,
                                   b->stream));
    return MM_OK;
}

void to_stats(const mm::DevState& s, double Mref, mm_stats* out) {
    const double EJ = kMu0 * Mref * Mref * 1e-27;
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

int status_of(int st) {
    switch (st) {
        case mm::ST_OK: return MM_OK;
        case mm::ST_NOT_CONVERGED: return MM_NOT_CONVERGED;
        case mm::ST_STALLED: return MM_STALLED;
        case mm::ST_NONFINITE: return MM_ERR_NONFINITE;
        case mm::ST_TIMEOUT: return MM_ERR_DEVICE_TIMEOUT;
        default: return MM_ERR_STATE;
    }
}

int sync_members(mm_batch* b) {
    for (auto& v : b->views) BK(cudaStreamSynchronize((cudaStream_t)v.stream));
    return MM_OK;
}

int check_errors(mm_batch* b) {
    std::vector<int> e((size_t)kErrWords * b->n);
    BK(cudaMemcpy(e.data(), b->d_err, e.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (int t = 0; t < b->n; ++t)
        if (e[(size_t)kErrWords * t]) return bfail(b, MM_ERR_DEVICE_TIMEOUT, "a device barrier wait ran out");
    return MM_OK;
}

}  // namespace

extern "C" {

int mm_batch_plan(int n, const int64_t* work, int total_blocks, double gamma, int32_t* blocks_out) {
    if (n < 1 || !work || !blocks_out || total_blocks < n || !(gamma >= 0.0)) return MM_ERR_ARG;
    std::vector<double> w(n);
    double sum = 0.0;
    for (int t = 0; t < n; ++t) {
        if (work[t] < 0) return MM_ERR_ARG;
        w[t] = std::pow((double)std::max<int64_t>(work[t], 1), gamma);
        sum += w[t];
    }
    std::vector<double> frac(n);
    int used = 0;
    for (int t = 0; t < n; ++t) {
        const double share = w[t] / sum * total_blocks;
        int k = (int)std::floor(share);
        if (k < 1) k = 1;
        blocks_out[t] = k;
        frac[t] = share - std::floor(share);
        used += k;
    }
    // hand out the remainder by largest fractional part (ties: lower index),
    // or take blocks back from the largest teams (ties: higher index)
    while (used < total_blocks) {
        int best = 0;
        for (int t = 1; t < n; ++t)
            if (frac[t] > frac[best]) best = t;
        blocks_out[best]++;
        frac[best] -= 1.0;
        ++used;
    }
    while (used > total_blocks) {
        int best = -1;
        for (int t = 0; t < n; ++t)
            if (blocks_out[t] > 1 && (best < 0 || blocks_out[t] >= blocks_out[best])) best = t;
        if (best < 0) return MM_ERR_ARG;
        blocks_out[best]--;
        --used;
    }
    return MM_OK;
}

int mm_batch_create(mm_batch** out, int n, mm_ctx* const* ctxs) {
    if (!out || n < 1 || !ctxs) return MM_ERR_ARG;
    *out = nullptr;
    mm_batch* b = new mm_batch();
    b->n = n;
    for (int t = 0; t < n; ++t) {
        mm::CtxView v;
        if (!ctxs[t] || mm::ctx_view(ctxs[t], &v) != MM_OK || !v.has_mesh) {
            delete b;
            return MM_ERR_STATE;
        }
        if (t > 0 && v.device != b->views[0].device) {
            delete b;
            return MM_ERR_ARG;
        }
        b->ctxs.push_back(ctxs[t]);
        b->views.push_back(v);
        b->work.push_back((int64_t)v.nnz_phi + v.nnz_mag + 8ll * v.nphi);
    }
    b->device = b->views[0].device;
    auto bail = [&](int code) {
        mm_batch_destroy(b);
        return code;
    };
    if (cudaSetDevice(b->device) != cudaSuccess) return bail(MM_ERR_CUDA);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(MM_ERR_CUDA);
    if (cudaMalloc(&b->d_probs, n * sizeof(mm::Problem)) != cudaSuccess) return bail(MM_ERR_OOM);
    if (cudaMalloc(&b->d_team_first, (n + 1) * sizeof(int)) != cudaSuccess) return bail(MM_ERR_OOM);
    if (cudaMalloc(&b->d_bar, (size_t)kBarWords * n * sizeof(unsigned)) != cudaSuccess) return bail(MM_ERR_OOM);
    if (cudaMalloc(&b->d_err, (size_t)kErrWords * n * sizeof(int)) != cudaSuccess) return bail(MM_ERR_OOM);
    if (cudaMalloc(&b->d_states, n * sizeof(mm::DevState*)) != cudaSuccess) return bail(MM_ERR_OOM);
    if (cudaMalloc(&b->d_stat, n * sizeof(mm::DevState)) != cudaSuccess) return bail(MM_ERR_OOM);
    if (cudaMallocHost(&b->h_stat, n * sizeof(mm::DevState)) != cudaSuccess) return bail(MM_ERR_OOM);
    std::vector<mm::DevState*> st(n);
    for (int t = 0; t < n; ++t) st[t] = b->views[t].d_state;
    if (cudaMemcpy(b->d_states, st.data(), n * sizeof(mm::DevState*), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(MM_ERR_CUDA);
    cudaEventCreate(&b->ev0);
    cudaEventCreate(&b->ev1);
    *out = b;
    return MM_OK;
}

void mm_batch_destroy(mm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    cudaFree(b->d_probs);
    cudaFree(b->d_team_first);
    cudaFree(b->d_part);
    cudaFree(b->d_bar);
    cudaFree(b->d_err);
    cudaFree(b->d_states);
    cudaFree(b->d_stat);
    if (b->h_stat) cudaFreeHost(b->h_stat);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* mm_batch_last_error(const mm_batch* b) { return b ? b->err.c_str() : "null batch"; }

int mm_batch_config(mm_batch* b, int blocks_per_sm, double gamma) {
    if (!b) return MM_ERR_ARG;
    if (blocks_per_sm < 2 || blocks_per_sm > 4) return bfail(b, MM_ERR_ARG, "blocks_per_sm must be 2, 3 or 4");
    if (!(gamma >= 0.0 && gamma <= 2.0)) return bfail(b, MM_ERR_ARG, "gamma must be in [0, 2]");
    b->variant = blocks_per_sm;
    b->gamma = gamma;
    return MM_OK;
}

int mm_batch_set_tiles(mm_batch* b, int32_t rows_per_thread, int32_t restrict_lanes) {
    if (!b) return MM_ERR_ARG;
    if (rows_per_thread < 0 || rows_per_thread > 2) return bfail(b, MM_ERR_ARG, "rows_per_thread must be 0, 1 or 2");
    if (restrict_lanes != 0 && restrict_lanes != 4 && restrict_lanes != 8 && restrict_lanes != 16)
        return bfail(b, MM_ERR_ARG, "restrict_lanes must be 0, 4, 8 or 16");
    b->tile_rows = rows_per_thread;
    b->restrict_lanes = restrict_lanes;
    return MM_OK;
}

int mm_batch_get_config(const mm_batch* b, int32_t* blocks_per_sm, double* gamma, int32_t* rows_per_thread,
                        int32_t* restrict_lanes) {
    if (!b) return MM_ERR_ARG;
    if (blocks_per_sm) *blocks_per_sm = b->variant;
    if (gamma) *gamma = b->gamma;
    if (rows_per_thread) *rows_per_thread = b->tile_rows == 1 ? 1 : 2;
    if (restrict_lanes) *restrict_lanes = (b->restrict_lanes == 4 || b->restrict_lanes == 16) ? b->restrict_lanes : 8;
    return MM_OK;
}

int mm_batch_minimize(mm_batch* b, const mm_params* p, mm_stats* stats_out) {
    if (!b) return MM_ERR_ARG;
    int rc;
    if ((rc = sync_members(b))) return rc;
    if ((rc = prepare(b, conv(p)))) return rc;
    BK(cudaEventRecord(b->ev0, b->stream));
    if ((rc = enqueue_launch(b))) return rc;
    BK(cudaEventRecord(b->ev1, b->stream));
    k_batch_status<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->n, b->d_states, b->d_stat);
    BK(cudaGetLastError());
    BK(cudaMemcpyAsync(b->h_stat, b->d_stat, b->n * sizeof(mm::DevState), cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    if ((rc = check_errors(b))) return rc;
    int first = MM_OK;
    for (int t = 0; t < b->n; ++t) {
        if (stats_out) to_stats(b->h_stat[t], b->views[t].Mref, &stats_out[t]);
        mm::ctx_refresh_state(b->ctxs[t]);
        const int s = status_of(b->h_stat[t].status);
        if (first == MM_OK && s != MM_OK) first = s;
    }
    return first;
}

int mm_batch_demag_curve(mm_batch* b, int64_t n_steps, const double* fields, const mm_params* p,
                         mm_stats* stats_out) {
    if (!b || n_steps < 1 || !fields) return MM_ERR_ARG;
    int rc;
    if ((rc = sync_members(b))) return rc;
    if ((rc = prepare(b, conv(p)))) return rc;
    const int n = b->n;
    std::vector<double> h((size_t)n_steps * n * 3);
    for (int64_t s = 0; s < n_steps; ++s)
        for (int t = 0; t < n; ++t)
            for (int c = 0; c < 3; ++c) {
                const double v = fields[((size_t)s * n + t) * 3 + c];
                if (!std::isfinite(v)) return bfail(b, MM_ERR_ARG, "non-finite field");
                h[((size_t)s * n + t) * 3 + c] = v / (kMu0 * b->views[t].Mref);
            }
    double* d_fields = nullptr;
    int* d_step = nullptr;
    mm::DevState* d_hist = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(d_fields);
        cudaFree(d_step);
        cudaFree(d_hist);
    };
    auto bail = [&](int code, const char* msg) {
        cleanup();
        return bfail(b, code, msg);
    };
    if (cudaMalloc(&d_fields, h.size() * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d_step, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&d_hist, (size_t)n_steps * n * sizeof(mm::DevState)) != cudaSuccess)
        return bail(MM_ERR_OOM, "device allocation failed");
    if (cudaMemcpy(d_fields, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(d_step, 0, sizeof(int)) != cudaSuccess)
        return bail(MM_ERR_CUDA, "upload failed");
    // one field step: set fields, clear barriers, solve every problem, record
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bail(MM_ERR_CUDA, "stream capture failed");
    k_batch_fields<<<(n + 127) / 128, 128, 0, b->stream>>>(n, d_fields, d_step, b->d_states);
    rc = enqueue_launch(b);
    k_batch_record<<<1, std::max(32, ((n + 31) / 32) * 32), 0, b->stream>>>(n, b->d_states, d_hist, d_step);
    cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
    if (rc || ce != cudaSuccess) return bail(MM_ERR_CUDA, "graph capture of the field step failed");
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) return bail(MM_ERR_CUDA, "graph instantiation failed");
    BK(cudaEventRecord(b->ev0, b->stream));
    for (int64_t s = 0; s < n_steps; ++s)
        if (cudaGraphLaunch(exec, b->stream) != cudaSuccess) return bail(MM_ERR_CUDA, "graph launch failed");
    BK(cudaEventRecord(b->ev1, b->stream));
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bail(MM_ERR_CUDA, "batch curve failed");
    if ((rc = check_errors(b))) {
        cleanup();
        return rc;
    }
    std::vector<mm::DevState> hist((size_t)n_steps * n);
    if (cudaMemcpy(hist.data(), d_hist, hist.size() * sizeof(mm::DevState), cudaMemcpyDeviceToHost) != cudaSuccess)
        return bail(MM_ERR_CUDA, "copy of the curve records failed");
    cleanup();
    int first = MM_OK;
    for (int64_t s = 0; s < n_steps; ++s)
        for (int t = 0; t < n; ++t) {
            const mm::DevState& d = hist[(size_t)s * n + t];
            if (stats_out) to_stats(d, b->views[t].Mref, &stats_out[(size_t)s * n + t]);
            const int st = status_of(d.status);
            if (first == MM_OK && st != MM_OK) first = st;
        }
    for (int t = 0; t < n; ++t) mm::ctx_refresh_state(b->ctxs[t]);
    return first;
}

int mm_batch_last_ms(mm_batch* b, double* ms) {
    if (!b || !ms) return MM_ERR_ARG;
    float f = 0.f;
    BK(cudaEventElapsedTime(&f, b->ev0, b->ev1));
    *ms = f;
    return MM_OK;
}

int mm_batch_autotune(mm_batch* b, const mm_params* p, int* chosen_blocks_per_sm, double* chosen_gamma,
                      double* best_ms) {
    if (!b) return MM_ERR_ARG;
    int rc;
    if ((rc = sync_members(b))) return rc;
    mm::Params prm = conv(p);
    prm.max_iter = std::min(prm.max_iter, 25);
    // save every member's state (current m and potential) to restore between trials
    const int n = b->n;
    std::vector<double*> saved_m(n, nullptr), saved_phi(n, nullptr);
    std::vector<mm::DevState> saved_state(n);
    auto release = [&]() {
        for (int t = 0; t < n; ++t) {
            cudaFree(saved_m[t]);
            cudaFree(saved_phi[t]);
        }
    };
    for (int t = 0; t < n; ++t) {
        const mm::CtxView& v = b->views[t];
        BK(cudaMemcpy(&saved_state[t], v.d_state, sizeof(mm::DevState), cudaMemcpyDeviceToHost));
        const size_t m3 = 3 * (size_t)v.nm;
        if (cudaMalloc(&saved_m[t], m3 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&saved_phi[t], (size_t)v.nphi * sizeof(double)) != cudaSuccess) {
            release();
            return bfail(b, MM_ERR_OOM, "autotune state copy failed");
        }
        BK(cudaMemcpy(saved_m[t], v.P->X[saved_state[t].cur], m3 * sizeof(double), cudaMemcpyDeviceToDevice));
        BK(cudaMemcpy(saved_phi[t], v.P->phi, (size_t)v.nphi * sizeof(double), cudaMemcpyDeviceToDevice));
    }
    auto restore = [&]() -> int {
        for (int t = 0; t < n; ++t) {
            const mm::CtxView& v = b->views[t];
            BK(cudaMemcpy(v.d_state, &saved_state[t], sizeof(mm::DevState), cudaMemcpyHostToDevice));
            BK(cudaMemcpy(v.P->X[saved_state[t].cur], saved_m[t], 3 * (size_t)v.nm * sizeof(double),
                          cudaMemcpyDeviceToDevice));
            BK(cudaMemcpy(v.P->phi, saved_phi[t], (size_t)v.nphi * sizeof(double), cudaMemcpyDeviceToDevice));
        }
        return MM_OK;
    };
    // One trial: the launch time of the current configuration (1e300 when it
    // does not fit), the members' states restored afterwards.
    auto trial = [&](double& ms) -> int {
        ms = 1e300;
        int r = prepare(b, prm);
        if (r == MM_ERR_ARG) return MM_OK;   // too many problems for this grid
        if (r) return r;
        BK(cudaEventRecord(b->ev0, b->stream));
        if ((r = enqueue_launch(b))) return r;
        BK(cudaEventRecord(b->ev1, b->stream));
        BK(cudaStreamSynchronize(b->stream));
        if ((r = check_errors(b))) return r;
        float t = 0.f;
        BK(cudaEventElapsedTime(&t, b->ev0, b->ev1));
        ms = t;
        return restore();
    };
    // Stage 1: kernel instantiation x team split at the default tile shape;
    // stage 2: the tile shape (rows per thread x restriction lanes) at the
    // best of stage 1.
    const int variants[3] = {2, 3, 4};
    const double gammas[3] = {0.5, 0.75, 1.0};
    const int rows[2] = {2, 1};
    const int lanes[3] = {8, 4, 16};
    double best = 1e300;
    int bv = b->variant, br = 0, bl = 0;
    double bg = b->gamma;
    b->tile_rows = 0;
    b->restrict_lanes = 0;
    for (int vi = 0; vi < 3; ++vi)
        for (int gi = 0; gi < 3; ++gi) {
            b->variant = variants[vi];
            b->gamma = gammas[gi];
            double ms;
            if ((rc = trial(ms))) {
                release();
                return rc;
            }
            if (ms < best) {
                best = ms;
                bv = variants[vi];
                bg = gammas[gi];
            }
        }
    if (best < 1e300) {
        b->variant = bv;
        b->gamma = bg;
        for (int ri = 0; ri < 2; ++ri)
            for (int li = 0; li < 3; ++li) {
                if (ri == 0 && li == 0) continue;   // the default shape, timed in stage 1
                b->tile_rows = rows[ri];
                b->restrict_lanes = lanes[li];
                double ms;
                if ((rc = trial(ms))) {
                    release();
                    return rc;
                }
                if (ms < best) {
                    best = ms;
                    br = rows[ri];
                    bl = lanes[li];
                }
            }
    }
    release();
    b->variant = bv;
    b->gamma = bg;
    b->tile_rows = br;
    b->restrict_lanes = bl;
    for (int t = 0; t < n; ++t) mm::ctx_refresh_state(b->ctxs[t]);
    if (chosen_blocks_per_sm) *chosen_blocks_per_sm = bv;
    if (chosen_gamma) *chosen_gamma = bg;
    if (best_ms) *best_ms = best;
    return best < 1e300 ? MM_OK : bfail(b, MM_ERR_ARG, "no configuration fits the batch");
}

}  // extern "C"
