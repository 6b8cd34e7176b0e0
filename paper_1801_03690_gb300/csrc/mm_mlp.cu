// Learned warm start (no counterpart in the paper): a per-node multilayer
// perceptron 16 -> 128 -> 128 -> 128 -> 4 (ReLU) that maps local features of
// a converged state and the next field increment to a correction of m and
// of the scalar potential.  Plain NCG then runs to t1-t3 from the corrected
// state, so the network only changes where the minimiser starts.
//
// The forward pass and the weight gradients run on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory: mm_mlp_tc.cuh);
// the same network on the warp-level mma.sync m16n8k16 path (BF16 operands,
// FP32 accumulation) is kept as a measured comparison
// (mm_mlp_set_tensor_path), and the activation-gradient kernel uses it:
//   k_mlp_forward   persistent; the weights (BF16, [out][in]) live in shared
//                   memory; inputs are standardised in FP32 (the network's
//                   own mean and 1/std) before the BF16 conversion, then each
//                   warp pushes 16 rows through all four layers
//                   (activations stay in shared memory; in training mode the
//                   hidden activations are also stored for the backward pass)
//   k_mlp_backward  per 16-row warp tile: dZ4 = 2 (Y - T) / (N n_out), then
//                   dA_{l-1} = dZ_l W_l and dZ_{l-1} = dA_{l-1} * [A_{l-1} > 0],
//                   storing every dZ_l
//   k_mlp_wgrad     split-K GEMM dW_l = dZ_l^T A_{l-1} over row chunks,
//                   partial tiles to global memory, then k_mlp_wreduce sums
//                   the partials in a fixed order (deterministic) and the
//                   bias gradients
//   k_mlp_adam      Adam on FP32 master weights, refreshes the BF16 copies
// Fragment layouts follow the PTX ISA description of mma.m16n8k16 (.bf16):
// with g = lane/4 and q = lane%4, A holds (g, 2q..2q+1), (g+8, 2q..), (g, 2q+8..),
// (g+8, 2q+8..); B holds (k = 2q..2q+1, n = g), (k = 2q+8.., n = g); C holds
// (g, 2q..2q+1), (g+8, 2q..2q+1).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/mmncg.h"
#include "mm_internal.cuh"

namespace {

constexpr int NIN = 16, NH = 128, NOUT = 4, NOUTP = 8;   // NOUTP: last layer padded to one n-tile
constexpr int LD1 = NIN + 8, LDH = NH + 8;                // padded shared-memory strides (bf16)
constexpr int WARPS = 4, ROWS_PER_BLOCK = 16 * WARPS;
constexpr int KCH = 128;                                  // rows per split-K chunk

// parameter layout (floats): W1 b1 W2 b2 W3 b3 W4 b4, W_l row-major [out][in]
constexpr int SZ_W1 = NH * NIN, SZ_W2 = NH * NH, SZ_W3 = NH * NH, SZ_W4 = NOUT * NH;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + SZ_W1;
constexpr int OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + SZ_W2;
constexpr int OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + SZ_W3;
constexpr int OFF_W4 = OFF_B3 + NH, OFF_B4 = OFF_W4 + SZ_W4;
constexpr int NPARAM = OFF_B4 + NOUT;

struct FwdSmem {
    __nv_bfloat16 w1[NH * LD1];
    __nv_bfloat16 w2[NH * LDH];
    __nv_bfloat16 w3[NH * LDH];
    __nv_bfloat16 w4[NOUTP * LDH];
    float b[3 * NH + NOUTP];
    float mean[NIN], istd[NIN];           // input standardisation (FP32)
    __nv_bfloat16 act[WARPS][16 * LDH];
    __nv_bfloat16 in[WARPS][16 * LD1];
};

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment of a row-major bf16 matrix (row stride ld) at (m0, k0).
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const __nv_bfloat16* A, int ld, int m0, int k0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const __nv_bfloat16* r0 = A + (m0 + g) * ld + k0 + 2 * q;
    const __nv_bfloat16* r1 = A + (m0 + g + 8) * ld + k0 + 2 * q;
    a[0] = pack2(r0[0], r0[1]);
    a[1] = pack2(r1[0], r1[1]);
    a[2] = pack2(r0[8], r0[9]);
    a[3] = pack2(r1[8], r1[9]);
}

// B fragment where element (k, n) is stored at Bt[n * ld + k] (k contiguous).
__device__ __forceinline__ void load_bt(uint32_t& b0, uint32_t& b1, const __nv_bfloat16* Bt, int ld, int k0,
                                        int n0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const __nv_bfloat16* r = Bt + (n0 + g) * ld + k0 + 2 * q;
    b0 = pack2(r[0], r[1]);
    b1 = pack2(r[8], r[9]);
}

// B fragment where element (k, n) is stored at B[k * ld + n] (n contiguous).
__device__ __forceinline__ void load_bn(uint32_t& b0, uint32_t& b1, const __nv_bfloat16* B, int ld, int k0,
                                        int n0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const __nv_bfloat16* c = B + (k0 + 2 * q) * ld + n0 + g;
    b0 = pack2(c[0], c[ld]);
    b1 = pack2(c[8 * ld], c[9 * ld]);
}

// A fragment where element (m, k) is stored at At[k * ld + m] (transposed).
__device__ __forceinline__ void load_at(uint32_t (&a)[4], const __nv_bfloat16* At, int ld, int m0, int k0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const __nv_bfloat16* c0 = At + (k0 + 2 * q) * ld + m0 + g;
    a[0] = pack2(c0[0], c0[ld]);
    a[1] = pack2(c0[8], c0[ld + 8]);
    a[2] = pack2(c0[8 * ld], c0[9 * ld]);
    a[3] = pack2(c0[8 * ld + 8], c0[9 * ld + 8]);
}

__device__ void load_weights(FwdSmem& s, const __nv_bfloat16* wb, const float* p, const float* norm) {
    for (int i = threadIdx.x; i < NIN; i += blockDim.x) {
        s.mean[i] = norm[i];
        s.istd[i] = norm[NIN + i];
    }
    for (int i = threadIdx.x; i < SZ_W1; i += blockDim.x) s.w1[(i / NIN) * LD1 + i % NIN] = wb[OFF_W1 + i];
    for (int i = threadIdx.x; i < SZ_W2; i += blockDim.x) s.w2[(i / NH) * LDH + i % NH] = wb[OFF_W2 + i];
    for (int i = threadIdx.x; i < SZ_W3; i += blockDim.x) s.w3[(i / NH) * LDH + i % NH] = wb[OFF_W3 + i];
    for (int i = threadIdx.x; i < NOUTP * NH; i += blockDim.x)
        s.w4[(i / NH) * LDH + i % NH] = (i < SZ_W4) ? wb[OFF_W4 + i] : __float2bfloat16(0.0f);
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        s.b[i] = p[OFF_B1 + i];
        s.b[NH + i] = p[OFF_B2 + i];
        s.b[2 * NH + i] = p[OFF_B3 + i];
    }
    for (int i = threadIdx.x; i < NOUTP; i += blockDim.x) s.b[3 * NH + i] = (i < NOUT) ? p[OFF_B4 + i] : 0.0f;
    __syncthreads();
}

// One hidden layer for the warp's 16 rows: act <- relu(act_in W^T + b), K = kin.
template <int KIN>
__device__ void hidden_layer(const __nv_bfloat16* ain, int lda, const __nv_bfloat16* W, int ldw, const float* b,
                             __nv_bfloat16* aout, __nv_bfloat16* gout, long long row0, long long n) {
    float c[NH / 8][4];
#pragma unroll
    for (int nt = 0; nt < NH / 8; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll
    for (int kt = 0; kt < KIN / 16; ++kt) {
        uint32_t a[4];
        load_a(a, ain, lda, 0, kt * 16);
#pragma unroll
        for (int nt = 0; nt < NH / 8; ++nt) {
            uint32_t b0, b1;
            load_bt(b0, b1, W, ldw, kt * 16, nt * 8);
            mma16816(c[nt], a, b0, b1);
        }
    }
    __syncwarp();
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NH / 8; ++nt) {
        const int col = nt * 8 + 2 * q;
        const __nv_bfloat16 v00 = __float2bfloat16(fmaxf(c[nt][0] + b[col], 0.0f));
        const __nv_bfloat16 v01 = __float2bfloat16(fmaxf(c[nt][1] + b[col + 1], 0.0f));
        const __nv_bfloat16 v10 = __float2bfloat16(fmaxf(c[nt][2] + b[col], 0.0f));
        const __nv_bfloat16 v11 = __float2bfloat16(fmaxf(c[nt][3] + b[col + 1], 0.0f));
        aout[g * LDH + col] = v00;
        aout[g * LDH + col + 1] = v01;
        aout[(g + 8) * LDH + col] = v10;
        aout[(g + 8) * LDH + col + 1] = v11;
        if (gout) {
            if (row0 + g < n) {
                gout[(row0 + g) * NH + col] = v00;
                gout[(row0 + g) * NH + col + 1] = v01;
            }
            if (row0 + g + 8 < n) {
                gout[(row0 + g + 8) * NH + col] = v10;
                gout[(row0 + g + 8) * NH + col + 1] = v11;
            }
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(WARPS * 32) k_mlp_forward(long long n, const float* __restrict__ X,
                                                            const __nv_bfloat16* __restrict__ wb,
                                                            const float* __restrict__ p,
                                                            const float* __restrict__ norm, float* __restrict__ Y,
                                                            __nv_bfloat16* A1, __nv_bfloat16* A2,
                                                            __nv_bfloat16* A3, __nv_bfloat16* X0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdSmem& s = *reinterpret_cast<FwdSmem*>(smem_raw);
    load_weights(s, wb, p, norm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const long long ntiles = (n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
    __nv_bfloat16* in = s.in[warp];
    __nv_bfloat16* act = s.act[warp];
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long row0 = tile * ROWS_PER_BLOCK + warp * 16;
        for (int i = lane; i < 16 * NIN; i += 32) {
            const long long r = row0 + i / NIN;
            const int c = i % NIN;
            const __nv_bfloat16 v = __float2bfloat16(r < n ? (X[r * NIN + c] - s.mean[c]) * s.istd[c] : 0.0f);
            in[(i / NIN) * LD1 + i % NIN] = v;
            if (X0 && r < n) X0[r * NIN + i % NIN] = v;
        }
        __syncwarp();
        hidden_layer<NIN>(in, LD1, s.w1, LD1, s.b, act, A1, row0, n);
        hidden_layer<NH>(act, LDH, s.w2, LDH, s.b + NH, act, A2, row0, n);
        hidden_layer<NH>(act, LDH, s.w3, LDH, s.b + 2 * NH, act, A3, row0, n);
        float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int kt = 0; kt < NH / 16; ++kt) {
            uint32_t a[4], b0, b1;
            load_a(a, act, LDH, 0, kt * 16);
            load_bt(b0, b1, s.w4, LDH, kt * 16, 0);
            mma16816(c, a, b0, b1);
        }
        const int col = 2 * q;
        if (col < NOUT) {
            if (row0 + g < n) {
                Y[(row0 + g) * NOUT + col] = c[0] + s.b[3 * NH + col];
                Y[(row0 + g) * NOUT + col + 1] = c[1] + s.b[3 * NH + col + 1];
            }
            if (row0 + g + 8 < n) {
                Y[(row0 + g + 8) * NOUT + col] = c[2] + s.b[3 * NH + col];
                Y[(row0 + g + 8) * NOUT + col + 1] = c[3] + s.b[3 * NH + col + 1];
            }
        }
        __syncwarp();
    }
}

struct BwdSmem {
    __nv_bfloat16 w2[NH * LDH];
    __nv_bfloat16 w3[NH * LDH];
    __nv_bfloat16 w4[16 * LDH];          // rows >= NOUT are zero
    __nv_bfloat16 dz[WARPS][16 * LDH];
};

// dA = dZ W for the warp's 16 rows (K = kout, N = 128), then
// dZ_prev = dA * [A_prev > 0]; writes dZ_prev to shared memory and global.
template <int KOUT>
__device__ void backward_layer(const __nv_bfloat16* dz, const __nv_bfloat16* W, const __nv_bfloat16* Aprev,
                               __nv_bfloat16* dzs, __nv_bfloat16* dzg, long long row0, long long n) {
    float c[NH / 8][4];
#pragma unroll
    for (int nt = 0; nt < NH / 8; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll
    for (int kt = 0; kt < KOUT / 16; ++kt) {
        uint32_t a[4];
        load_a(a, dz, LDH, 0, kt * 16);
#pragma unroll
        for (int nt = 0; nt < NH / 8; ++nt) {
            uint32_t b0, b1;
            load_bn(b0, b1, W, LDH, kt * 16, nt * 8);     // (k = out, n = in) = W[out][in]
            mma16816(c[nt], a, b0, b1);
        }
    }
    __syncwarp();
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NH / 8; ++nt) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long r = row0 + g + 8 * h;
            const int col = nt * 8 + 2 * q;
            float v0 = c[nt][2 * h], v1 = c[nt][2 * h + 1];
            if (r < n) {
                if (!(__bfloat162float(Aprev[r * NH + col]) > 0.0f)) v0 = 0.0f;
                if (!(__bfloat162float(Aprev[r * NH + col + 1]) > 0.0f)) v1 = 0.0f;
            } else {
                v0 = v1 = 0.0f;
            }
            const __nv_bfloat16 b0 = __float2bfloat16(v0), b1 = __float2bfloat16(v1);
            dzs[(g + 8 * h) * LDH + col] = b0;
            dzs[(g + 8 * h) * LDH + col + 1] = b1;
            if (r < n) {
                dzg[r * NH + col] = b0;
                dzg[r * NH + col + 1] = b1;
            }
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(WARPS * 32) k_mlp_backward(long long n, const float* __restrict__ Y,
                                                             const float* __restrict__ T,
                                                             const __nv_bfloat16* __restrict__ wb,
                                                             const __nv_bfloat16* A1, const __nv_bfloat16* A2,
                                                             const __nv_bfloat16* A3, __nv_bfloat16* DZ4,
                                                             __nv_bfloat16* DZ3, __nv_bfloat16* DZ2,
                                                             __nv_bfloat16* DZ1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem& s = *reinterpret_cast<BwdSmem*>(smem_raw);
    for (int i = threadIdx.x; i < SZ_W2; i += blockDim.x) s.w2[(i / NH) * LDH + i % NH] = wb[OFF_W2 + i];
    for (int i = threadIdx.x; i < SZ_W3; i += blockDim.x) s.w3[(i / NH) * LDH + i % NH] = wb[OFF_W3 + i];
    for (int i = threadIdx.x; i < 16 * NH; i += blockDim.x)
        s.w4[(i / NH) * LDH + i % NH] = (i < SZ_W4) ? wb[OFF_W4 + i] : __float2bfloat16(0.0f);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float scale = 2.0f / ((float)n * (float)NOUT);
    __nv_bfloat16* dz = s.dz[warp];
    const long long ntiles = (n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long row0 = tile * ROWS_PER_BLOCK + warp * 16;
        // dZ4 [16 x 16] (columns >= NOUT zero)
        for (int i = lane; i < 16 * 16; i += 32) {
            const int rr = i / 16, cc = i % 16;
            const long long r = row0 + rr;
            float v = 0.0f;
            if (r < n && cc < NOUT) v = scale * (Y[r * NOUT + cc] - T[r * NOUT + cc]);
            const __nv_bfloat16 bv = __float2bfloat16(v);
            dz[rr * LDH + cc] = bv;
            if (r < n && cc < NOUT) DZ4[r * NOUT + cc] = bv;
        }
        __syncwarp();
        backward_layer<16>(dz, s.w4, A3, dz, DZ3, row0, n);
        backward_layer<NH>(dz, s.w3, A2, dz, DZ2, row0, n);
        backward_layer<NH>(dz, s.w2, A1, dz, DZ1, row0, n);
    }
}

// Split-K weight gradient: partial[chunk][o][i] = sum over the chunk's rows
// of DZ[r][o] * A[r][i] for o < nout, i < nin (nout padded to 16, nin to 16).
__global__ void __launch_bounds__(WARPS * 32) k_mlp_wgrad(long long n, int nout, int nin,
                                                          const __nv_bfloat16* __restrict__ DZ,
                                                          const __nv_bfloat16* __restrict__ A,
                                                          float* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldz = 128 + 8, lda = 128 + 8;
    __nv_bfloat16* dzs = reinterpret_cast<__nv_bfloat16*>(smem_raw);           // [KCH][ldz]
    __nv_bfloat16* as = dzs + KCH * ldz;                                          // [KCH][lda]
    const long long r0 = (long long)blockIdx.x * KCH;
    const int mp = (nout + 15) / 16 * 16, np = (nin + 15) / 16 * 16;
    for (int i = threadIdx.x; i < KCH * mp; i += blockDim.x) {
        const int rr = i / mp, o = i % mp;
        const long long r = r0 + rr;
        dzs[rr * ldz + o] = (r < n && o < nout) ? DZ[r * nout + o] : __float2bfloat16(0.0f);
    }
    for (int i = threadIdx.x; i < KCH * np; i += blockDim.x) {
        const int rr = i / np, c = i % np;
        const long long r = r0 + rr;
        as[rr * lda + c] = (r < n && c < nin) ? A[r * nin + c] : __float2bfloat16(0.0f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int mtiles = mp / 16, ntiles = np / 8;
    float* out = partial + (size_t)blockIdx.x * nout * nin;
    // warp w takes m-tiles w, w + WARPS, ...
    for (int mt = warp; mt < mtiles; mt += WARPS) {
        for (int nt0 = 0; nt0 < ntiles; nt0 += 8) {
            float c[8][4];
#pragma unroll
            for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0f;
#pragma unroll
            for (int kt = 0; kt < KCH / 16; ++kt) {
                uint32_t a[4];
                load_at(a, dzs, ldz, mt * 16, kt * 16);        // (m = out, k = row) = DZ[row][out]
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (nt0 + j < ntiles) {
                        uint32_t b0, b1;
                        load_bn(b0, b1, as, lda, kt * 16, (nt0 + j) * 8);   // (k = row, n = in)
                        mma16816(c[j], a, b0, b1);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (nt0 + j >= ntiles) continue;
                const int col = (nt0 + j) * 8 + 2 * q;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int o = mt * 16 + g + 8 * h;
                    if (o < nout) {
                        if (col < nin) out[o * nin + col] = c[j][2 * h];
                        if (col + 1 < nin) out[o * nin + col + 1] = c[j][2 * h + 1];
                    }
                }
            }
        }
    }
}

// grad_W[e] = sum over chunks (ascending) of partial[chunk][e]; bias
// gradients grad_b[o] = sum over rows (ascending) of DZ[r][o].
__global__ void k_mlp_wreduce(int nchunks, int nw, const float* __restrict__ partial, float* __restrict__ gw) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nw) return;
    float s = 0.0f;
    for (int c = 0; c < nchunks; ++c) s += partial[(size_t)c * nw + e];
    gw[e] = s;
}

__global__ void k_mlp_bgrad(long long n, int nout, const __nv_bfloat16* __restrict__ DZ, float* __restrict__ gb) {
    // one block per output column, fixed-order tree
    __shared__ float sh[256];
    const int o = blockIdx.x;
    float s = 0.0f;
    for (long long r = threadIdx.x; r < n; r += blockDim.x) s += __bfloat162float(DZ[r * nout + o]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[o] = sh[0];
}

__global__ void k_mlp_loss(long long n, const float* __restrict__ Y, const float* __restrict__ T, float* out) {
    __shared__ float sh[256];
    float s = 0.0f;
    for (long long i = threadIdx.x; i < n * NOUT; i += blockDim.x) {
        const float d = Y[i] - T[i];
        s += d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / ((float)n * NOUT);
}

__global__ void k_mlp_adam(int np, float* p, const float* g, float* m, float* v, __nv_bfloat16* wb, float lr,
                           float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    wb[i] = __float2bfloat16(w);
}

__global__ void k_to_bf16(int n, const float* a, __nv_bfloat16* b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(a[i]);
}

// Features of magnetic node i from a converged state (internal units):
// m, effective field, exchange field, anisotropy field, field increment and
// the scalar potential.
__global__ void k_features(int nm, const mm::Problem* Pp, const mm::DevState* st, double dh0, double dh1,
                           double dh2, float* X) {
    const mm::Problem& P = *Pp;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    const int s = st->cur;
    const double* x = P.X[s];
    const long long nz = P.nnzm;
    const int sl = i >> 5;
    const long long base = P.m_sptr[sl] + (i & 31);
    const int width = (int)((P.m_sptr[sl + 1] - P.m_sptr[sl]) >> 5);
    double c0 = 0, c1 = 0, c2 = 0, t0 = 0, t1 = 0, t2 = 0;
    for (int k = 0; k < width; ++k) {
        const long long e = base + 32ll * k;
        const int j = P.m_col[e];
        const double ka = P.KA[e];
        c0 += ka * x[j];
        c1 += ka * x[nm + j];
        c2 += ka * x[2 * nm + j];
        const double ph = P.phi[j];
        t0 += P.G[e] * ph;
        t1 += P.G[nz + e] * ph;
        t2 += P.G[2 * nz + e] * ph;
    }
    const double m0 = x[i], m1 = x[nm + i], m2 = x[2 * nm + i];
    const double kxx = P.CK[i], kxy = P.CK[nm + i], kxz = P.CK[2 * nm + i];
    const double kyy = P.CK[3 * nm + i], kyz = P.CK[4 * nm + i], kzz = P.CK[5 * nm + i];
    const double iw = 1.0 / P.w[i];
    const double ex0 = -2.0 * c0 * iw, ex1 = -2.0 * c1 * iw, ex2 = -2.0 * c2 * iw;
    const double an0 = -(kxx * m0 + kxy * m1 + kxz * m2) * iw;
    const double an1 = -(kxy * m0 + kyy * m1 + kyz * m2) * iw;
    const double an2 = -(kxz * m0 + kyz * m1 + kzz * m2) * iw;
    const double he0 = ex0 + an0 - t0 * iw + st->h[0];
    const double he1 = ex1 + an1 - t1 * iw + st->h[1];
    const double he2 = ex2 + an2 - t2 * iw + st->h[2];
    float* f = X + (size_t)i * NIN;
    f[0] = (float)m0;
    f[1] = (float)m1;
    f[2] = (float)m2;
    f[3] = (float)he0;
    f[4] = (float)he1;
    f[5] = (float)he2;
    f[6] = (float)ex0;
    f[7] = (float)ex1;
    f[8] = (float)ex2;
    f[9] = (float)an0;
    f[10] = (float)an1;
    f[11] = (float)an2;
    f[12] = (float)dh0;
    f[13] = (float)dh1;
    f[14] = (float)dh2;
    f[15] = (float)P.phi[i];
}

// Largest predicted nodal change max_i |sm |dh| y_i[0:3]| (non-negative
// floats compare like their bit patterns).
__global__ void k_apply_max(int nm, const float* Y, double sm, double dhn, unsigned* mx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    const float* y = Y + (size_t)i * NOUT;
    const float d = (float)(sm * dhn * sqrt((double)y[0] * y[0] + (double)y[1] * y[1] + (double)y[2] * y[2]));
    if (isfinite(d)) atomicMax(mx, __float_as_uint(d));
}

// m_i <- N(m_i + c sm |dh| y_i[0:3]);  phi_i += c sphi |dh| y_i[3] (magnetic
// rows), c = min(1, cap / max_i |predicted change|).
__global__ void k_apply(int nm, const mm::Problem* Pp, const mm::DevState* st, const float* Y, double sm,
                        double sphi, double dhn, double cap, const unsigned* mx) {
    const mm::Problem& P = *Pp;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    const double big = (double)__uint_as_float(*mx);
    const double c = (cap > 0.0 && big > cap) ? cap / big : 1.0;
    double* x = P.X[st->cur];
    const float* y = Y + (size_t)i * NOUT;
    const double u0 = x[i] + c * sm * dhn * y[0];
    const double u1 = x[nm + i] + c * sm * dhn * y[1];
    const double u2 = x[2 * nm + i] + c * sm * dhn * y[2];
    const double r = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
    if (r > 0.0 && isfinite(r)) {
        x[i] = u0 / r;
        x[nm + i] = u1 / r;
        x[2 * nm + i] = u2 / r;
    }
    const double dp = c * sphi * dhn * y[3];
    if (isfinite(dp)) P.phi[i] += dp;
}

}  // namespace

// Training targets from two consecutive converged states' features (rows
// of X0 at field k, X1 at field k+1): T_i = (m_{k+1} - m_k, phi_{k+1} -
// phi_k) / |dh| (features 0..2 are m, 15 the potential); the largest nodal
// change |m_{k+1} - m_k| goes to mx (non-negative floats compare like their
// bit patterns).
__global__ void k_ws_targets(long long n, const float* __restrict__ X0, const float* __restrict__ X1, float inv_dh,
                             float* __restrict__ T, unsigned* mx) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float c = 0.0f;
    if (i < n) {
        const float* a = X0 + i * NIN;
        const float* b = X1 + i * NIN;
        const float d0 = b[0] - a[0], d1 = b[1] - a[1], d2 = b[2] - a[2];
        T[i * NOUT] = d0 * inv_dh;
        T[i * NOUT + 1] = d1 * inv_dh;
        T[i * NOUT + 2] = d2 * inv_dh;
        T[i * NOUT + 3] = (b[15] - a[15]) * inv_dh;
        c = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    }
    for (int o = 16; o > 0; o >>= 1) c = fmaxf(c, __shfl_down_sync(0xffffffffu, c, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, __float_as_uint(c));
}

// Column statistics of an [n][w] float array (columns c0 .. c0+nc-1, or all
// nc columns pooled when pool = 1): FP64 sums per block in a fixed order,
// written to part[block][2 * nc]: sum of x - shift and of (x - shift)^2.
__global__ void k_colstats(long long n, int w, int c0, int nc, int pool, const float* __restrict__ X,
                           const double* __restrict__ shift, double* __restrict__ part) {
    __shared__ double sh[2][16][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < nc; ++c) {
        double s1 = 0.0, s2 = 0.0;
        const double sc = shift[pool ? 0 : c];
        for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
            if (pool) {
                for (int q = 0; q < nc; ++q) {
                    const double x = (double)X[r * w + c0 + q] - sc;
                    s1 += x;
                    s2 += x * x;
                }
            } else {
                const double x = (double)X[r * w + c0 + c] - sc;
                s1 += x;
                s2 += x * x;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            sh[0][c][warp] = s1;
            sh[1][c][warp] = s2;
        }
        if (pool) break;
    }
    __syncthreads();
    const int nout = pool ? 1 : nc;
    if (threadIdx.x < nout) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            a += sh[0][threadIdx.x][q];
            b += sh[1][threadIdx.x][q];
        }
        part[(size_t)blockIdx.x * 2 * nout + threadIdx.x] = a;
        part[(size_t)blockIdx.x * 2 * nout + nout + threadIdx.x] = b;
    }
}

__global__ void k_scale_targets(long long n, const float* __restrict__ T, float sm, float sp, float* __restrict__ Tn) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Tn[i * NOUT] = T[i * NOUT] / sm;
    Tn[i * NOUT + 1] = T[i * NOUT + 1] / sm;
    Tn[i * NOUT + 2] = T[i * NOUT + 2] / sm;
    Tn[i * NOUT + 3] = T[i * NOUT + 3] / sp;
}

#include "mm_mlp_tc.cuh"

struct mm_mlp {
    int device = 0;
    int nsm = 0;
    float* p = nullptr;           // FP32 master parameters
    float* norm = nullptr;        // input standardisation: mean[16], 1/std[16]
    __nv_bfloat16* wb = nullptr;  // BF16 copy
    float* g = nullptr;           // gradients
    float* am = nullptr;          // Adam moments
    float* av = nullptr;
    long long step = 0;
    // work buffers (grown on demand)
    long long cap = 0;
    __nv_bfloat16 *X0 = nullptr, *A1 = nullptr, *A2 = nullptr, *A3 = nullptr;
    __nv_bfloat16 *DZ1 = nullptr, *DZ2 = nullptr, *DZ3 = nullptr, *DZ4 = nullptr;
    float* Yb = nullptr;
    float* part = nullptr;
    float* loss = nullptr;
    cudaStream_t stream = nullptr;
    // inference buffers for the warm start
    long long fcap = 0;
    float *F = nullptr, *FY = nullptr;
    mm::Problem* d_prob = nullptr;
    unsigned* d_max = nullptr;
    int* d_err = nullptr;         // set by a tensor-core wait that ran out
    int path = 0;                 // 0: tcgen05 forward pass, 1: mma.sync (comparison)
};

namespace {

#define MK(call)                                         \
    do {                                                 \
        if ((call) != cudaSuccess) {                     \
            cudaGetLastError();                          \
            return MM_ERR_CUDA;                          \
        }                                                \
    } while (0)

size_t fwd_smem() { return sizeof(FwdSmem); }
size_t bwd_smem() { return sizeof(BwdSmem); }
size_t wgrad_smem() { return (size_t)2 * KCH * (128 + 8) * sizeof(__nv_bfloat16); }

int ensure(mm_mlp* M, long long n) {
    if (n <= M->cap) return MM_OK;
    cudaFree(M->X0);
    cudaFree(M->A1);
    cudaFree(M->A2);
    cudaFree(M->A3);
    cudaFree(M->DZ1);
    cudaFree(M->DZ2);
    cudaFree(M->DZ3);
    cudaFree(M->DZ4);
    cudaFree(M->Yb);
    cudaFree(M->part);
    const long long nch = (n + KCH - 1) / KCH;
    if (cudaMalloc(&M->X0, n * NIN * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&M->A1, n * NH * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&M->A2, n * NH * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&M->A3, n * NH * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&M->DZ1, n * NH * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&M->DZ2, n * NH * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&M->DZ3, n * NH * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&M->DZ4, n * NOUT * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&M->Yb, n * NOUT * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&M->part, (size_t)nch * NH * NH * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        M->cap = 0;
        return MM_ERR_OOM;
    }
    M->cap = n;
    return MM_OK;
}

int launch_forward(mm_mlp* M, const float* X, long long n, float* Y, bool train) {
    if (M->path == 0) {
        const int grid = std::max(1, std::min((int)((n + tc::TM - 1) / tc::TM), 2 * M->nsm));
        tc::k_mlp_forward_tc<<<grid, tc::TM, sizeof(tc::Smem), M->stream>>>(
            n, X, M->wb, M->p, M->norm, Y, train ? M->A1 : nullptr, train ? M->A2 : nullptr,
            train ? M->A3 : nullptr, train ? M->X0 : nullptr, M->d_err);
        MK(cudaGetLastError());
        return MM_OK;
    }
    const int grid = std::max(1, std::min((int)((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK), 2 * M->nsm));
    k_mlp_forward<<<grid, WARPS * 32, fwd_smem(), M->stream>>>(n, X, M->wb, M->p, M->norm, Y, train ? M->A1 : nullptr,
                                                               train ? M->A2 : nullptr, train ? M->A3 : nullptr,
                                                               train ? M->X0 : nullptr);
    MK(cudaGetLastError());
    return MM_OK;
}

// forward + backward into M->g (no update)
int gradient(mm_mlp* M, const float* X, const float* T, long long n) {
    int rc;
    if ((rc = ensure(M, n))) return rc;
    if ((rc = launch_forward(M, X, n, M->Yb, true))) return rc;
    const int grid = std::max(1, std::min((int)((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK), 2 * M->nsm));
    k_mlp_backward<<<grid, WARPS * 32, bwd_smem(), M->stream>>>(n, M->Yb, T, M->wb, M->A1, M->A2, M->A3, M->DZ4,
                                                                M->DZ3, M->DZ2, M->DZ1);
    MK(cudaGetLastError());
    const int nch = (int)((n + KCH - 1) / KCH);
    struct L {
        int nout, nin, offw, offb;
        const __nv_bfloat16 *dz, *a;
    } layers[4] = {{NH, NIN, OFF_W1, OFF_B1, M->DZ1, M->X0},
                   {NH, NH, OFF_W2, OFF_B2, M->DZ2, M->A1},
                   {NH, NH, OFF_W3, OFF_B3, M->DZ3, M->A2},
                   {NOUT, NH, OFF_W4, OFF_B4, M->DZ4, M->A3}};
    for (auto& l : layers) {
        if (M->path == 0)
            tc::k_mlp_wgrad_tc<<<nch, tc::TM, sizeof(tc::WgSmem), M->stream>>>(n, l.nout, l.nin, l.dz, l.a, M->part,
                                                                              M->d_err);
        else
            k_mlp_wgrad<<<nch, WARPS * 32, wgrad_smem(), M->stream>>>(n, l.nout, l.nin, l.dz, l.a, M->part);
        MK(cudaGetLastError());
        const int nw = l.nout * l.nin;
        k_mlp_wreduce<<<(nw + 255) / 256, 256, 0, M->stream>>>(nch, nw, M->part, M->g + l.offw);
        k_mlp_bgrad<<<l.nout, 256, 0, M->stream>>>(n, l.nout, l.dz, M->g + l.offb);
        MK(cudaGetLastError());
    }
    return MM_OK;
}

// MM_ERR_DEVICE_TIMEOUT if a tensor-core wait of the last launches ran out
// (the flag is cleared); call after synchronising the stream.
int check_err(mm_mlp* M) {
    int e = 0;
    MK(cudaMemcpy(&e, M->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!e) return MM_OK;
    MK(cudaMemset(M->d_err, 0, sizeof(int)));
    return MM_ERR_DEVICE_TIMEOUT;
}

}  // namespace

extern "C" {

int64_t mm_mlp_param_count(void) { return NPARAM; }

int mm_mlp_set_tensor_path(mm_mlp* M, int path) {
    if (!M || (path != 0 && path != 1)) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    MK(cudaStreamSynchronize(M->stream));
    M->path = path;
    return MM_OK;
}

int mm_mlp_create(mm_mlp** out, int device, uint64_t seed) {
    if (!out) return MM_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return MM_ERR_CUDA;
    mm_mlp* M = new mm_mlp();
    M->device = device;
    cudaDeviceGetAttribute(&M->nsm, cudaDevAttrMultiProcessorCount, device);
    auto bail = [&](int code) {
        mm_mlp_destroy(M);
        return code;
    };
    if (cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(MM_ERR_CUDA);
    if (cudaMalloc(&M->p, NPARAM * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&M->wb, NPARAM * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&M->g, NPARAM * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&M->am, NPARAM * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&M->av, NPARAM * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&M->loss, sizeof(float)) != cudaSuccess || cudaMalloc(&M->d_prob, sizeof(mm::Problem)) != cudaSuccess ||
        cudaMalloc(&M->norm, 2 * NIN * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&M->d_max, sizeof(unsigned)) != cudaSuccess || cudaMalloc(&M->d_err, sizeof(int)) != cudaSuccess)
        return bail(MM_ERR_OOM);
    if (cudaMemset(M->d_err, 0, sizeof(int)) != cudaSuccess) return bail(MM_ERR_CUDA);
    {
        float id[2 * NIN];
        for (int i = 0; i < NIN; ++i) {
            id[i] = 0.0f;
            id[NIN + i] = 1.0f;
        }
        if (cudaMemcpy(M->norm, id, sizeof(id), cudaMemcpyHostToDevice) != cudaSuccess) return bail(MM_ERR_CUDA);
    }
    if (cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem()) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem()) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem()) !=
            cudaSuccess ||
        cudaFuncSetAttribute(tc::k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(tc::Smem)) != cudaSuccess ||
        cudaFuncSetAttribute(tc::k_mlp_forward_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100) !=
            cudaSuccess ||
        cudaFuncSetAttribute(tc::k_mlp_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(tc::WgSmem)) != cudaSuccess)
        return bail(MM_ERR_CUDA);
    // He-uniform initialisation (host RNG, seeded), zero biases
    std::vector<float> h(NPARAM, 0.0f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int nout, int nin) {
        std::uniform_real_distribution<float> u(-std::sqrt(6.0f / nin), std::sqrt(6.0f / nin));
        for (int i = 0; i < nout * nin; ++i) h[off + i] = u(rng);
    };
    fill(OFF_W1, NH, NIN);
    fill(OFF_W2, NH, NH);
    fill(OFF_W3, NH, NH);
    fill(OFF_W4, NOUT, NH);
    *out = M;
    return mm_mlp_set_params(M, h.data(), NPARAM);
}

void mm_mlp_destroy(mm_mlp* M) {
    if (!M) return;
    cudaSetDevice(M->device);
    if (M->stream) cudaStreamSynchronize(M->stream);
    for (void* q : {(void*)M->p, (void*)M->norm, (void*)M->wb, (void*)M->g, (void*)M->am, (void*)M->av, (void*)M->loss,
                    (void*)M->X0, (void*)M->A1, (void*)M->A2, (void*)M->A3, (void*)M->DZ1, (void*)M->DZ2,
                    (void*)M->DZ3, (void*)M->DZ4, (void*)M->Yb, (void*)M->part, (void*)M->F, (void*)M->FY,
                    (void*)M->d_prob, (void*)M->d_max, (void*)M->d_err})
        if (q) cudaFree(q);
    if (M->stream) cudaStreamDestroy(M->stream);
    delete M;
}

int mm_mlp_set_params(mm_mlp* M, const float* params, int64_t count) {
    if (!M || !params || count != NPARAM) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    MK(cudaMemcpy(M->p, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    k_to_bf16<<<(NPARAM + 255) / 256, 256, 0, M->stream>>>(NPARAM, M->p, M->wb);
    MK(cudaMemsetAsync(M->am, 0, NPARAM * sizeof(float), M->stream));
    MK(cudaMemsetAsync(M->av, 0, NPARAM * sizeof(float), M->stream));
    MK(cudaStreamSynchronize(M->stream));
    M->step = 0;
    return MM_OK;
}

int mm_mlp_set_input_norm(mm_mlp* M, const float* mean, const float* stdev) {
    if (!M || !mean || !stdev) return MM_ERR_ARG;
    float h[2 * NIN];
    for (int i = 0; i < NIN; ++i) {
        if (!(stdev[i] > 0.0f) || !std::isfinite(mean[i])) return MM_ERR_ARG;
        h[i] = mean[i];
        h[NIN + i] = 1.0f / stdev[i];
    }
    MK(cudaSetDevice(M->device));
    MK(cudaStreamSynchronize(M->stream));
    MK(cudaMemcpy(M->norm, h, sizeof(h), cudaMemcpyHostToDevice));
    return MM_OK;
}

int mm_mlp_get_params(mm_mlp* M, float* params, int64_t count) {
    if (!M || !params || count != NPARAM) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    MK(cudaStreamSynchronize(M->stream));
    MK(cudaMemcpy(params, M->p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return MM_OK;
}

int mm_mlp_forward(mm_mlp* M, const float* X_dev, int64_t n, float* Y_dev) {
    if (!M || !X_dev || !Y_dev || n < 1) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    int rc = launch_forward(M, X_dev, n, Y_dev, false);
    if (rc) return rc;
    MK(cudaStreamSynchronize(M->stream));
    return check_err(M);
}

int mm_mlp_gradient(mm_mlp* M, const float* X_dev, const float* T_dev, int64_t n, float* grad_host,
                    float* loss_out) {
    if (!M || !X_dev || !T_dev || n < 1) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    int rc = gradient(M, X_dev, T_dev, n);
    if (rc) return rc;
    k_mlp_loss<<<1, 256, 0, M->stream>>>(n, M->Yb, T_dev, M->loss);
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(M->stream));
    if ((rc = check_err(M))) return rc;
    if (grad_host) MK(cudaMemcpy(grad_host, M->g, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss_out) MK(cudaMemcpy(loss_out, M->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return MM_OK;
}

int mm_mlp_train_step(mm_mlp* M, const float* X_dev, const float* T_dev, int64_t n, float lr, float* loss_out) {
    if (!M || !X_dev || !T_dev || n < 1 || !(lr > 0.0f)) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    int rc = gradient(M, X_dev, T_dev, n);
    if (rc) return rc;
    M->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)M->step), c2 = 1.0f - std::pow(b2, (float)M->step);
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, M->stream>>>(NPARAM, M->p, M->g, M->am, M->av, M->wb, lr, b1, b2,
                                                             1e-8f, c1, c2);
    MK(cudaGetLastError());
    if (loss_out) {
        k_mlp_loss<<<1, 256, 0, M->stream>>>(n, M->Yb, T_dev, M->loss);
        MK(cudaGetLastError());
        MK(cudaMemcpyAsync(loss_out, M->loss, sizeof(float), cudaMemcpyDeviceToHost, M->stream));
        MK(cudaStreamSynchronize(M->stream));
        if ((rc = check_err(M))) return rc;
    }
    return MM_OK;
}

}  // extern "C"

namespace {

// Mean and unbiased standard deviation of columns c0 .. c0+nc-1 of an [n][w]
// device array (pool = 1: all nc columns together), FP64, two passes (the
// second about the first pass's mean), blocks reduced in a fixed order.
int col_mean_std(mm_mlp* M, const float* X, long long n, int w, int c0, int nc, int pool, double* mean,
                 double* sd) {
    const int nb = std::max(1, std::min((int)((n + 255) / 256), 4 * M->nsm));
    const int nout = pool ? 1 : nc;
    double *dpart = nullptr, *dshift = nullptr;
    MK(cudaMalloc(&dpart, (size_t)nb * 2 * nout * sizeof(double)));
    if (cudaMalloc(&dshift, 16 * sizeof(double)) != cudaSuccess) {
        cudaFree(dpart);
        return MM_ERR_OOM;
    }
    std::vector<double> shift(16, 0.0), part((size_t)nb * 2 * nout);
    const double cnt = (double)n * (pool ? nc : 1);
    int rc = MM_OK;
    for (int pass = 0; pass < 2 && rc == MM_OK; ++pass) {
        if (cudaMemcpy(dshift, shift.data(), 16 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = MM_ERR_CUDA;
            break;
        }
        k_colstats<<<nb, 256, 0, M->stream>>>(n, w, c0, nc, pool, X, dshift, dpart);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(M->stream) != cudaSuccess ||
            cudaMemcpy(part.data(), dpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = MM_ERR_CUDA;
            break;
        }
        for (int c = 0; c < nout; ++c) {
            double s1 = 0.0, s2 = 0.0;
            for (int b = 0; b < nb; ++b) {
                s1 += part[(size_t)b * 2 * nout + c];
                s2 += part[(size_t)b * 2 * nout + nout + c];
            }
            if (pass == 0) {
                shift[c] = s1 / cnt;                       // the mean
            } else {
                mean[c] = shift[c] + s1 / cnt;
                sd[c] = cnt > 1 ? std::sqrt(std::max(0.0, (s2 - s1 * s1 / cnt) / (cnt - 1.0))) : 0.0;
            }
        }
    }
    cudaFree(dpart);
    cudaFree(dshift);
    return rc;
}

}  // namespace

extern "C" {

int mm_mlp_fit_input_norm(mm_mlp* M, const float* X_dev, int64_t n) {
    if (!M || !X_dev || n < 2) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    MK(cudaStreamSynchronize(M->stream));
    double mean[NIN], sd[NIN];
    int rc = col_mean_std(M, X_dev, n, NIN, 0, NIN, 0, mean, sd);
    if (rc) return rc;
    float h[2 * NIN];
    for (int i = 0; i < NIN; ++i) {
        if (!std::isfinite(mean[i]) || !std::isfinite(sd[i])) return MM_ERR_NONFINITE;
        const double s = (sd[i] > 1e-6 * (std::fabs(mean[i]) + 1.0)) ? sd[i] : 1.0;   // constant: centre only
        h[i] = (float)mean[i];
        h[NIN + i] = (float)(1.0 / s);
    }
    MK(cudaMemcpy(M->norm, h, sizeof(h), cudaMemcpyHostToDevice));
    return MM_OK;
}

int mm_mlp_get_input_norm(mm_mlp* M, float* mean, float* inv_stdev) {
    if (!M || !mean || !inv_stdev) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    MK(cudaStreamSynchronize(M->stream));
    float h[2 * NIN];
    MK(cudaMemcpy(h, M->norm, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < NIN; ++i) {
        mean[i] = h[i];
        inv_stdev[i] = h[NIN + i];
    }
    return MM_OK;
}

int mm_mlp_fit_target_scales(mm_mlp* M, const float* T_dev, int64_t n, float* Tn_dev, double* scale_m,
                             double* scale_phi) {
    if (!M || !T_dev || !Tn_dev || !scale_m || !scale_phi || n < 2) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    MK(cudaStreamSynchronize(M->stream));
    double mm_[1], sm[1], mp[1], sp[1];
    int rc = col_mean_std(M, T_dev, n, NOUT, 0, 3, 1, mm_, sm);
    if (rc) return rc;
    if ((rc = col_mean_std(M, T_dev, n, NOUT, 3, 1, 0, mp, sp))) return rc;
    if (!std::isfinite(sm[0]) || !std::isfinite(sp[0])) return MM_ERR_NONFINITE;
    *scale_m = std::max(sm[0], 1e-12);
    *scale_phi = std::max(sp[0], 1e-12);
    k_scale_targets<<<(unsigned)((n + 255) / 256), 256, 0, M->stream>>>(n, T_dev, (float)*scale_m, (float)*scale_phi,
                                                                       Tn_dev);
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(M->stream));
    return MM_OK;
}

int mm_warmstart_targets(mm_mlp* M, const float* X0_dev, const float* X1_dev, int64_t n, float* T_dev,
                         double* dh_out, double* max_change_out) {
    if (!M || !X0_dev || !X1_dev || !T_dev || !dh_out || !max_change_out || n < 1) return MM_ERR_ARG;
    MK(cudaSetDevice(M->device));
    MK(cudaStreamSynchronize(M->stream));
    float inc[3];
    MK(cudaMemcpy(inc, X0_dev + 12, 3 * sizeof(float), cudaMemcpyDeviceToHost));   // the field increment
    const double dh = std::sqrt((double)inc[0] * inc[0] + (double)inc[1] * inc[1] + (double)inc[2] * inc[2]);
    *dh_out = dh;
    *max_change_out = 0.0;
    if (!(dh > 0.0)) return MM_OK;
    MK(cudaMemsetAsync(M->d_max, 0, sizeof(unsigned), M->stream));
    k_ws_targets<<<(unsigned)((n + 255) / 256), 256, 0, M->stream>>>(n, X0_dev, X1_dev, (float)(1.0 / dh), T_dev,
                                                                     M->d_max);
    MK(cudaGetLastError());
    unsigned mx = 0;
    MK(cudaMemcpyAsync(&mx, M->d_max, sizeof(unsigned), cudaMemcpyDeviceToHost, M->stream));
    MK(cudaStreamSynchronize(M->stream));
    float f;
    std::memcpy(&f, &mx, sizeof(f));
    *max_change_out = f;
    return MM_OK;
}

int mm_warmstart_features(mm_ctx* ctx, const double mu0h_next[3], float* X_dev) {
    mm::CtxView v;
    if (!ctx || !mu0h_next || !X_dev || mm::ctx_view(ctx, &v) != MM_OK) return MM_ERR_ARG;
    if (!v.has_mesh) return mm::ctx_fail(ctx, MM_ERR_STATE, "no mesh uploaded");
    MK(cudaSetDevice(v.device));
    cudaStream_t st = (cudaStream_t)v.stream;
    MK(cudaStreamSynchronize(st));
    mm::Problem* dp = nullptr;
    MK(cudaMalloc(&dp, sizeof(mm::Problem)));
    cudaMemcpy(dp, v.P, sizeof(mm::Problem), cudaMemcpyHostToDevice);
    mm::DevState hs;
    cudaMemcpy(&hs, v.d_state, sizeof(mm::DevState), cudaMemcpyDeviceToHost);
    const double s = 1.0 / (4e-7 * 3.14159265358979323846 * v.Mref);
    k_features<<<(v.nm + 255) / 256, 256, 0, st>>>(v.nm, dp, v.d_state, mu0h_next[0] * s - hs.h[0],
                                                   mu0h_next[1] * s - hs.h[1], mu0h_next[2] * s - hs.h[2], X_dev);
    const cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(st);
    cudaFree(dp);
    return e == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}

int mm_warmstart_apply(mm_ctx* ctx, mm_mlp* M, const double mu0h_next[3], double scale_m, double scale_phi,
                       double max_change) {
    mm::CtxView v;
    if (!ctx || !M || !mu0h_next || mm::ctx_view(ctx, &v) != MM_OK) return MM_ERR_ARG;
    if (!v.has_mesh) return mm::ctx_fail(ctx, MM_ERR_STATE, "no mesh uploaded");
    MK(cudaSetDevice(v.device));
    if (v.nm > M->fcap) {
        cudaFree(M->F);
        cudaFree(M->FY);
        M->F = M->FY = nullptr;
        MK(cudaMalloc(&M->F, (size_t)v.nm * NIN * sizeof(float)));
        MK(cudaMalloc(&M->FY, (size_t)v.nm * NOUT * sizeof(float)));
        M->fcap = v.nm;
    }
    int rc = mm_warmstart_features(ctx, mu0h_next, M->F);
    if (rc) return rc;
    if ((rc = launch_forward(M, M->F, v.nm, M->FY, false))) return rc;
    MK(cudaStreamSynchronize(M->stream));
    if ((rc = check_err(M))) return mm::ctx_fail(ctx, rc, "a tensor-core wait of the network ran out");
    mm::DevState hs;
    MK(cudaMemcpy(&hs, v.d_state, sizeof(mm::DevState), cudaMemcpyDeviceToHost));
    const double s = 1.0 / (4e-7 * 3.14159265358979323846 * v.Mref);
    const double d0 = mu0h_next[0] * s - hs.h[0], d1 = mu0h_next[1] * s - hs.h[1], d2 = mu0h_next[2] * s - hs.h[2];
    const double dhn = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    MK(cudaMemcpy(M->d_prob, v.P, sizeof(mm::Problem), cudaMemcpyHostToDevice));
    cudaStream_t st = (cudaStream_t)v.stream;
    MK(cudaMemsetAsync(M->d_max, 0, sizeof(unsigned), st));
    k_apply_max<<<(v.nm + 255) / 256, 256, 0, st>>>(v.nm, M->FY, scale_m, dhn, M->d_max);
    k_apply<<<(v.nm + 255) / 256, 256, 0, st>>>(v.nm, M->d_prob, v.d_state, M->FY, scale_m, scale_phi, dhn,
                                                max_change, M->d_max);
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(st));
    return MM_OK;
}

}  // extern "C"
