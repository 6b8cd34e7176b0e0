// Forward pass and weight gradient of the warm-start network on the
// 5th-generation tensor cores (tcgen05): BF16 operands staged in shared
// memory, FP32 accumulators in tensor memory (TMEM), M = 128 per MMA (one
// TMEM lane per row).  Included by mm_mlp.cu (it uses that file's layer
// sizes and parameter layout).
//
// Per tile of 128 rows (4 warps, thread t owns row t of the tile):
//   x   = bf16((X - mean) / std)                  -> shared memory
//   h1  = relu(x W1^T + b1)   1 MMA  (K = 16)     TMEM -> registers -> bf16 -> shared
//   h2  = relu(h1 W2^T + b2)  8 MMAs (K = 8 x 16)
//   h3  = relu(h2 W3^T + b3)  8 MMAs
//   y   = h3 W4^T + b4        8 MMAs, N = 16 (outputs 4..15 are zero weights)
// One thread issues the MMAs of a layer and commits them to an mbarrier;
// every thread waits on it (bounded: a wait that runs out sets the error
// flag, and the block leaves after freeing its TMEM), then reads its row of
// the accumulator with tcgen05.ld.  The rounding points (input, weights,
// hidden activations to BF16; FP32 accumulation) are those of the mma.sync
// path, so both paths compute the same network.
//
// Operand layout in shared memory: "no swizzle, K-major" core matrices of
// 8 rows x 16 bytes (8 bf16 along K); element (r, k) of an R x K operand at
// byte (r / 8) * (16 K) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, i.e.
// core matrices 128 B apart along K (the descriptor's leading-dimension
// offset) and 16 K bytes apart along R (its stride-dimension offset).  The
// weights W_l [out][in] are the B operands as stored (K = in contiguous).
#pragma once

namespace tc {

constexpr int TM = 128;      // rows per tile = the MMA's M = TMEM lanes
constexpr int N4 = 16;       // the last layer's N, padded
constexpr int TCOLS = 128;   // TMEM columns allocated (one N = 128 accumulator)
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per MMA wait

struct __align__(128) Smem {
    __nv_bfloat16 w1[NH * NIN];
    __nv_bfloat16 w2[NH * NH];
    __nv_bfloat16 w3[NH * NH];
    __nv_bfloat16 w4[N4 * NH];
    __nv_bfloat16 x[TM * NIN];
    __nv_bfloat16 h[TM * NH];
    float b[3 * NH + N4];
    float mean[NIN], istd[NIN];
    unsigned long long bar;
    unsigned tmem;
};

__device__ __forceinline__ unsigned core_off(int r, int k, int K) {
    return (unsigned)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading-dimension offset
// 128 B (next core matrix along K), stride-dimension offset 16 K B (next 8
// rows), the descriptor version bits 46-48 = 0b001, no swizzle.
__device__ __forceinline__ unsigned long long sdesc(const void* p, int K) {
    const unsigned long long a = (smem_u32(p) & 0x3FFFFu) >> 4;
    const unsigned long long lbo = 128u >> 4, sbo = (unsigned)(K * 16) >> 4;
    return a | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(unsigned tmem, unsigned long long a, unsigned long long b, unsigned id,
                                    unsigned accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate));
}

__device__ __forceinline__ void commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the completion of the mbarrier phase with the given parity;
// false if it did not complete within kWaitNs.
__device__ __forceinline__ bool wait_phase(unsigned long long* bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    const unsigned long long t0 = now_ns();
    while (true) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (now_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Hidden-layer epilogue of this thread's row: h = relu(acc + b) to BF16,
// into the next layer's A operand (shared) and, in training, to global
// memory (row-major [n][128], as the backward pass reads it).
__device__ __forceinline__ void hidden_epilogue(Smem& s, unsigned tlane, const float* b, int row, long long r,
                                                long long n, __nv_bfloat16* gout) {
#pragma unroll 1
    for (int j = 0; j < NH / 32; ++j) {
        float v[32];
        tmem_ld32(tlane + 32 * j, v);
        __align__(16) __nv_bfloat16 o[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) o[i] = __float2bfloat16(fmaxf(v[i] + b[32 * j + i], 0.0f));
        unsigned char* hb = reinterpret_cast<unsigned char*>(s.h);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(hb + core_off(row, 32 * j + 8 * q, NH)) = reinterpret_cast<const uint4*>(o)[q];
        if (gout && r < n) {
            uint4* g = reinterpret_cast<uint4*>(gout + r * NH + 32 * j);
#pragma unroll
            for (int q = 0; q < 4; ++q) g[q] = reinterpret_cast<const uint4*>(o)[q];
        }
    }
}

// Two CTAs per SM (2 x 110 KB of shared memory, 2 x 128 TMEM columns): while
// one waits on its MMAs or runs its epilogue, the other's MMAs run.
__global__ void __launch_bounds__(TM, 2) k_mlp_forward_tc(long long n, const float* __restrict__ X,
                                                           const __nv_bfloat16* __restrict__ wb,
                                                           const float* __restrict__ p,
                                                           const float* __restrict__ norm, float* __restrict__ Y,
                                                           __nv_bfloat16* A1, __nv_bfloat16* A2, __nv_bfloat16* A3,
                                                           __nv_bfloat16* X0, int* err) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    Smem& s = *reinterpret_cast<Smem*>(tc_smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    // weights (BF16 copies) into the core-matrix layout, biases, standardisation
    unsigned char* w1 = reinterpret_cast<unsigned char*>(s.w1);
    unsigned char* w2 = reinterpret_cast<unsigned char*>(s.w2);
    unsigned char* w3 = reinterpret_cast<unsigned char*>(s.w3);
    unsigned char* w4 = reinterpret_cast<unsigned char*>(s.w4);
    for (int i = tid; i < SZ_W1; i += TM)
        *reinterpret_cast<__nv_bfloat16*>(w1 + core_off(i / NIN, i % NIN, NIN)) = wb[OFF_W1 + i];
    for (int i = tid; i < SZ_W2; i += TM) {
        *reinterpret_cast<__nv_bfloat16*>(w2 + core_off(i / NH, i % NH, NH)) = wb[OFF_W2 + i];
        *reinterpret_cast<__nv_bfloat16*>(w3 + core_off(i / NH, i % NH, NH)) = wb[OFF_W3 + i];
    }
    for (int i = tid; i < N4 * NH; i += TM)
        *reinterpret_cast<__nv_bfloat16*>(w4 + core_off(i / NH, i % NH, NH)) =
            (i < SZ_W4) ? wb[OFF_W4 + i] : __float2bfloat16(0.0f);
    for (int i = tid; i < NH; i += TM) {
        s.b[i] = p[OFF_B1 + i];
        s.b[NH + i] = p[OFF_B2 + i];
        s.b[2 * NH + i] = p[OFF_B3 + i];
    }
    if (tid < N4) s.b[3 * NH + tid] = (tid < NOUT) ? p[OFF_B4 + tid] : 0.0f;
    if (tid < NIN) {
        s.mean[tid] = norm[tid];
        s.istd[tid] = norm[NIN + tid];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    before_sync();
    __syncthreads();
    after_sync();
    const unsigned tbase = s.tmem;
    const unsigned tlane = tbase + ((unsigned)(warp * 32) << 16);   // this warp's 32 TMEM lanes
    const unsigned long long dx = sdesc(s.x, NIN), dh = sdesc(s.h, NH);
    const unsigned long long dw1 = sdesc(s.w1, NIN), dw2 = sdesc(s.w2, NH), dw3 = sdesc(s.w3, NH),
                             dw4 = sdesc(s.w4, NH);
    constexpr unsigned id128 = idesc_bf16(TM, NH), id16 = idesc_bf16(TM, N4);
    // one K step of 16 bf16 = two core matrices = 256 B = 16 in the address field
    constexpr unsigned long long KSTEP = 256 >> 4;
    unsigned parity = 0;
    bool ok = true;
    const long long ntiles = (n + TM - 1) / TM;
    auto layer_done = [&]() -> bool {        // the layer's MMAs have completed (all threads agree)
        const bool mine = wait_phase(&s.bar, parity);
        const bool all = __syncthreads_and(mine) != 0;
        if (all) parity ^= 1u;
        after_sync();
        return all;
    };
    auto before_mma = [&]() {
        fence_async_smem();
        before_sync();
        __syncthreads();
        after_sync();
    };
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long r = tile * TM + tid;
        unsigned char* xb = reinterpret_cast<unsigned char*>(s.x);
#pragma unroll
        for (int c = 0; c < NIN; ++c) {
            const __nv_bfloat16 v = __float2bfloat16(r < n ? (X[r * NIN + c] - s.mean[c]) * s.istd[c] : 0.0f);
            *reinterpret_cast<__nv_bfloat16*>(xb + core_off(tid, c, NIN)) = v;
            if (X0 && r < n) X0[r * NIN + c] = v;
        }
        before_mma();
        if (tid == 0) {
            mma(tbase, dx, dw1, id128, 0u);
            commit(&s.bar);
        }
        if (!(ok = layer_done())) break;
        hidden_epilogue(s, tlane, s.b, tid, r, n, A1);
        before_mma();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < NH / 16; ++k) mma(tbase, dh + k * KSTEP, dw2 + k * KSTEP, id128, k > 0);
            commit(&s.bar);
        }
        if (!(ok = layer_done())) break;
        hidden_epilogue(s, tlane, s.b + NH, tid, r, n, A2);
        before_mma();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < NH / 16; ++k) mma(tbase, dh + k * KSTEP, dw3 + k * KSTEP, id128, k > 0);
            commit(&s.bar);
        }
        if (!(ok = layer_done())) break;
        hidden_epilogue(s, tlane, s.b + 2 * NH, tid, r, n, A3);
        before_mma();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < NH / 16; ++k) mma(tbase, dh + k * KSTEP, dw4 + k * KSTEP, id16, k > 0);
            commit(&s.bar);
        }
        if (!(ok = layer_done())) break;
        float v[16];
        tmem_ld16(tlane, v);
        if (r < n) {
#pragma unroll
            for (int c = 0; c < NOUT; ++c) Y[r * NOUT + c] = v[c] + s.b[3 * NH + c];
        }
        before_sync();
        __syncthreads();                  // TMEM read before the next tile's first MMA overwrites it
        after_sync();
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        wait_phase(&s.bar, parity);       // the phase that did not complete: let it finish (bounded)
    }
    before_sync();
    __syncthreads();
    after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TCOLS) : "memory");
}

// ---- weight gradient on tcgen05.  Chunk c of KW = 128 rows gives the
// partial dW = dZ^T A_prev over its rows as one MMA product of M = 128
// (outputs; zero rows beyond nout), N = nin padded to 16, K = 128 (rows):
// both operands are staged transposed (dZ^T: (out, row), A_prev^T: (in,
// row)) into the K-major core-matrix layout, 8 MMAs of K = 16 accumulate in
// TMEM, and the epilogue writes partial[c][o][i] (o < nout, i < nin) for the
// fixed-order reduction over chunks that follows.
constexpr int KW = 128;

struct __align__(128) WgSmem {
    __nv_bfloat16 a[TM * KW];
    __nv_bfloat16 b[TM * KW];
    unsigned long long bar;
    unsigned tmem;
};

__global__ void __launch_bounds__(TM, 2) k_mlp_wgrad_tc(long long n, int nout, int nin,
                                                         const __nv_bfloat16* __restrict__ DZ,
                                                         const __nv_bfloat16* __restrict__ A,
                                                         float* __restrict__ partial, int* err) {
    extern __shared__ __align__(1024) unsigned char tc_wsmem[];
    WgSmem& s = *reinterpret_cast<WgSmem*>(tc_wsmem);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int np = (nin + 15) / 16 * 16;
    const long long r = (long long)blockIdx.x * KW + tid;     // this thread's row of the chunk
    unsigned char* ab = reinterpret_cast<unsigned char*>(s.a);
    unsigned char* bb = reinterpret_cast<unsigned char*>(s.b);
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    for (int o = 0; o < TM; ++o)
        *reinterpret_cast<__nv_bfloat16*>(ab + core_off(o, tid, KW)) =
            (r < n && o < nout) ? DZ[r * nout + o] : zero;
    for (int i = 0; i < np; ++i)
        *reinterpret_cast<__nv_bfloat16*>(bb + core_off(i, tid, KW)) = (r < n && i < nin) ? A[r * nin + i] : zero;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    before_sync();
    __syncthreads();
    after_sync();
    const unsigned tbase = s.tmem;
    const unsigned tlane = tbase + ((unsigned)(warp * 32) << 16);
    constexpr unsigned long long KSTEP = 256 >> 4;
    if (tid == 0) {
        const unsigned long long da = sdesc(s.a, KW), db = sdesc(s.b, KW);
        const unsigned id = idesc_bf16(TM, np);
#pragma unroll
        for (int k = 0; k < KW / 16; ++k) mma(tbase, da + k * KSTEP, db + k * KSTEP, id, k > 0);
        commit(&s.bar);
    }
    const bool ok = __syncthreads_and(wait_phase(&s.bar, 0u)) != 0;
    after_sync();
    if (ok) {
        float* out = partial + (size_t)blockIdx.x * nout * nin;
        const int o = tid;                                     // TMEM lane = output row
        if (np == 16) {
            float v[16];
            tmem_ld16(tlane, v);
            if (o < nout)
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (i < nin) out[o * nin + i] = v[i];
        } else {
#pragma unroll 1
            for (int j = 0; j < np / 32; ++j) {
                float v[32];
                tmem_ld32(tlane + 32 * j, v);
                if (o < nout)
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (32 * j + i < nin) out[o * nin + 32 * j + i] = v[i];
            }
        }
    } else {
        if (tid == 0) atomicExch(err, 1);
        wait_phase(&s.bar, 0u);
    }
    before_sync();
    __syncthreads();
    after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TCOLS) : "memory");
}

}  // namespace tc
