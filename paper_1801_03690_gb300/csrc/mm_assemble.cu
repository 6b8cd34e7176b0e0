// GPU assembly of the operators of Eq. (energy) (Sec. 2.2) on P1 tetrahedra.
//
// k_tet_geometry: per tetrahedron, the volume and the gradients of the four
//   barycentric hat functions.  With edges e_k = x_k - x_0 (k = 1..3) and
//   det = e_1 . (e_2 x e_3), the gradients are
//   grad lam_1 = (e_2 x e_3)/det, grad lam_2 = (e_3 x e_1)/det,
//   grad lam_3 = (e_1 x e_2)/det, grad lam_0 = -(sum of the three), and the
//   volume is |det|/6.  Coordinates are converted from metres to nm.
// k_assemble_phi / k_assemble_mag: one thread per matrix row gathers the
//   contributions of the row's incident tetrahedra in ascending tet order
//   (no floating-point atomics, so assembly is deterministic) into the
//   row's SELL-32 slots:
//     K_phi[p][q]  += V b_p . b_q                      (all tets)
//     K_A[i][j]    += A V b_i . b_j                    (magnetic tets)
//     G[i][j]      += Ms V/4 b_j      (= D_{j i}, used for D^T phi)
//     B[i][j]      += Ms V/4 b_i      (= D_{i j}, used for D m)
//     C_K[i]       += -2 K V/4 k k^T,  w_i += Ms V/4    (lumped)
//   Material constants are converted to internal units:
//   Ms/Mref, A/(mu0 Mref^2 nm^2), K/(mu0 Mref^2).
#include <cuda_runtime.h>
#include <math.h>

#include "mm_assemble.cuh"

namespace mm {

namespace {
constexpr double kMu0 = 4e-7 * 3.14159265358979323846;
constexpr double kNm = 1e-9;
}

__global__ void k_tet_geometry(int64_t nt, const double* __restrict__ xyz, const int* __restrict__ tets,
                               double* __restrict__ vol, double* __restrict__ grad, int* __restrict__ bad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt) return;
    double x[4][3];
    for (int v = 0; v < 4; ++v) {
        const int n = tets[4 * e + v];
        for (int c = 0; c < 3; ++c) x[v][c] = xyz[3 * (int64_t)n + c] / kNm;
    }
    double a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = x[1][k] - x[0][k];
        b[k] = x[2][k] - x[0][k];
        c[k] = x[3][k] - x[0][k];
    }
    const double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    const double ca[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
    const double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double det = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
    if (!(fabs(det) > 0.0) || !isfinite(det)) {
        atomicExch(bad, 1);
        vol[e] = 0.0;
        for (int k = 0; k < 12; ++k) grad[12 * e + k] = 0.0;
        return;
    }
    vol[e] = fabs(det) / 6.0;
    double* g = grad + 12 * e;
    for (int k = 0; k < 3; ++k) {
        const double g1 = bc[k] / det, g2 = ca[k] / det, g3 = ab[k] / det;
        g[3 + k] = g1;
        g[6 + k] = g2;
        g[9 + k] = g3;
        g[k] = -(g1 + g2 + g3);
    }
}

__device__ __forceinline__ int find_slot(const int* col, long long base, int width, int target) {
    for (int k = 0; k < width; ++k)
        if (col[base + 32ll * k] == target) return k;
    return -1;
}

__global__ void k_assemble_phi(AssembleArgs A) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.nphi) return;
    const int s = p >> 5;
    const long long base = A.p_sptr[s] + (p & 31);
    const int width = (int)((A.p_sptr[s + 1] - A.p_sptr[s]) >> 5);
    for (int k = 0; k < width; ++k) A.Kp[base + 32ll * k] = 0.0;
    if (A.phi_ident[p]) {
        const int k = find_slot(A.p_col, base, width, p);
        if (k >= 0) A.Kp[base + 32ll * k] = 1.0;
        A.dinvP[p] = 1.0;
        return;
    }
    const int n = A.node_of_phi[p];
    for (long long q = A.nt_ptr[n]; q < A.nt_ptr[n + 1]; ++q) {
        const int e = A.nt_idx[q];
        int lr = 0;
        while (A.tets[4ll * e + lr] != n) ++lr;
        const double V = A.vol[e];
        const double* g = A.grad + 12ll * e;
        for (int lc = 0; lc < 4; ++lc) {
            const int pc = A.phi_of[A.tets[4ll * e + lc]];
            if (pc < 0 || A.phi_ident[pc]) continue;
            const int k = find_slot(A.p_col, base, width, pc);
            if (k < 0) {
                atomicExch(A.bad, 2);
                continue;
            }
            const double bb = g[3 * lr] * g[3 * lc] + g[3 * lr + 1] * g[3 * lc + 1] + g[3 * lr + 2] * g[3 * lc + 2];
            A.Kp[base + 32ll * k] += V * bb;
        }
    }
    const int kd = find_slot(A.p_col, base, width, p);
    const double dg = (kd >= 0) ? A.Kp[base + 32ll * kd] : 0.0;
    A.dinvP[p] = (dg > 0.0) ? 1.0 / dg : 1.0;
    if (!(dg > 0.0)) atomicExch(A.bad, 3);
}

__global__ void k_assemble_mag(AssembleArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.nm) return;
    const int s = i >> 5;
    const long long base = A.m_sptr[s] + (i & 31);
    const int width = (int)((A.m_sptr[s + 1] - A.m_sptr[s]) >> 5);
    const long long nz = A.nnzm;
    for (int k = 0; k < width; ++k) {
        const long long e = base + 32ll * k;
        A.KA[e] = 0.0;
        for (int c = 0; c < 3; ++c) {
            A.G[c * nz + e] = 0.0;
            A.B[c * nz + e] = 0.0;
        }
    }
    double ck[6] = {0, 0, 0, 0, 0, 0};
    double w = 0.0;
    const double mu0M2 = kMu0 * A.Mref * A.Mref;
    const int n = A.mag_nodes[i];
    const bool rhs_row = !A.phi_ident[i];
    for (long long q = A.nt_ptr[n]; q < A.nt_ptr[n + 1]; ++q) {
        const int e = A.nt_idx[q];
        const int r = A.region[e];
        const double* mat = A.materials + 6 * r;
        if (!(mat[0] > 0.0)) continue;                      // non-magnetic tet
        const double Ms = mat[0] / A.Mref;
        const double Aex = mat[1] / (mu0M2 * kNm * kNm);
        const double K = mat[2] / mu0M2;
        const double an = sqrt(mat[3] * mat[3] + mat[4] * mat[4] + mat[5] * mat[5]);
        const double kx = mat[3] / an, ky = mat[4] / an, kz = mat[5] / an;
        int lr = 0;
        while (A.tets[4ll * e + lr] != n) ++lr;
        const double V = A.vol[e];
        const double* g = A.grad + 12ll * e;
        const double q4 = Ms * V / 4.0;
        for (int lc = 0; lc < 4; ++lc) {
            const int j = A.mag_of[A.tets[4ll * e + lc]];
            const int k = find_slot(A.m_col, base, width, j);
            if (k < 0) {
                atomicExch(A.bad, 4);
                continue;
            }
            const long long slot = base + 32ll * k;
            const double bb = g[3 * lr] * g[3 * lc] + g[3 * lr + 1] * g[3 * lc + 1] + g[3 * lr + 2] * g[3 * lc + 2];
            A.KA[slot] += Aex * V * bb;
            for (int c = 0; c < 3; ++c) {
                A.G[c * nz + slot] += q4 * g[3 * lc + c];
                if (rhs_row) A.B[c * nz + slot] += q4 * g[3 * lr + c];
            }
        }
        const double kq = -2.0 * K * V / 4.0;
        ck[0] += kq * kx * kx;
        ck[1] += kq * kx * ky;
        ck[2] += kq * kx * kz;
        ck[3] += kq * ky * ky;
        ck[4] += kq * ky * kz;
        ck[5] += kq * kz * kz;
        w += Ms * V / 4.0;
    }
    for (int c = 0; c < 6; ++c) A.CK[c * A.nm + i] = ck[c];
    A.w[i] = w;
    const int kd = find_slot(A.m_col, base, width, i);
    const double dg = (kd >= 0) ? 2.0 * A.KA[base + 32ll * kd] : 0.0;
    A.dinvA[i] = (dg != 0.0) ? 1.0 / dg : 1.0;
}

}  // namespace mm
