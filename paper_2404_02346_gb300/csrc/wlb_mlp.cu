// Learned surrogate of the radiation force: MLP 4 -> 256 -> 256 -> 256 -> 1
// (GELU hidden layers, linear output) trained on forces from the batched
// lattice runs.  Not part of the paper's method: it maps (k a, k z0, kappa~,
// c~) to the normalised force and is judged by the lattice runs.
//
// Every matrix product runs on the 5th-generation tensor cores: BF16 operands
// are staged in shared memory in the canonical K-major layout without swizzle
// (8-row x 16-byte core matrices), one thread issues tcgen05.mma (kind::f16,
// M = 128, N <= 256, K = 16 per instruction) into an FP32 accumulator in
// tensor memory, completion is signalled through an mbarrier, and the four
// warps read the accumulator back with tcgen05.ld for a fused epilogue.
// Weights are kept as FP32 masters (Adam) with BF16 copies in both
// orientations for the forward and backward products.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/wlb.h"

namespace {

constexpr int kIn = 4, kHid = 256, kInPad = 16, kOutPad = 16;
constexpr int kTileM = 128, kKC = 64;
constexpr int kSmemBytes = 96 * 1024;  // >= tiles; also caps residency at 2 CTAs/SM (TMEM 2 x 256 cols)
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitLimit = 1LL << 22;

// Packed parameter offsets (FP32): W1 (256x4), b1, W2 (256x256), b2, W3, b3, W4 (1x256), b4.
constexpr int oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid, oW3 = ob2 + kHid,
              ob3 = oW3 + kHid * kHid, oW4 = ob3 + kHid, ob4 = oW4 + kHid, kParams = ob4 + 1;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets >> 4, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *mbar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait: false if the phase did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase) {
    for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_try(mbar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// tcgen05.ld of 32 columns without the wait, and the wait that completes it:
// the wait names the destination registers, so no read of them moves above it.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Inputs are mapped to [-1, 1] by the training box before the BF16 rounding.
__device__ __forceinline__ float normalise_input(float x, float lo, float hi) {
    return 2.0f * (x - lo) / (hi - lo) - 1.0f;
}

__device__ __forceinline__ float rcp_approx(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float ex2_approx(float v) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// GELU(z) = z Phi(z), with Phi from the rational-times-exponential form of
// Abramowitz & Stegun 7.1.26 (|error in erf| <= 1.5e-7): for x = |z| / sqrt 2
// and t = 1 / (1 + p x), q = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2) / 2
// equals Phi(-|z|), and z Phi(z) = z / 2 + |z| (1/2 - q) for either sign (no
// branch).  The halving is folded into the coefficients (exact in binary).
// gelu2 below evaluates it for two values at once; every kernel calls it, so
// all paths evaluate the same bits.
constexpr float kAS_p = 0.3275911f, kAS_a1 = 0.254829592f, kAS_a2 = -0.284496736f, kAS_a3 = 1.421413741f,
                kAS_a4 = -1.453152027f, kAS_a5 = 1.061405429f;

// Packed pairs of FP32 values (Blackwell's f32x2 arithmetic: each lane is
// rounded exactly as the scalar instruction rounds it).
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The GELU above for two pre-activations at once, as the epilogue of every
// forward path evaluates it: the products and sums on packed pairs, |z| and
// the two MUFU steps per lane, about 9 instructions per value against 14 one
// value at a time.  Each packed instruction alone rounds every lane as its
// scalar form does, but the compiler contracts some packed products into the
// following packed sum (a fused multiply-add, one rounding fewer) although
// the instructions carry .rn; so the result can differ from the scalar
// sequence in the last place (about one negative input in 30), well inside
// the A&S bound.  Every path calls this one, so the paths agree bit for bit.
__device__ __forceinline__ void gelu2(float z0, float z1, float &g0, float &g1) {
    const unsigned long long z = f2_pack(z0, z1);
    const unsigned long long az = f2_pack(fabsf(z0), fabsf(z1));
    const float cp = kAS_p * 0.70710678118654752f;
    float u0, u1;
    f2_unpack(f2_fma(f2_pack(cp, cp), az, f2_pack(1.0f, 1.0f)), u0, u1);
    const unsigned long long t = f2_pack(rcp_approx(u0), rcp_approx(u1));
    unsigned long long p = f2_fma(f2_pack(0.5f * kAS_a5, 0.5f * kAS_a5), t, f2_pack(0.5f * kAS_a4, 0.5f * kAS_a4));
    p = f2_fma(p, t, f2_pack(0.5f * kAS_a3, 0.5f * kAS_a3));
    p = f2_fma(p, t, f2_pack(0.5f * kAS_a2, 0.5f * kAS_a2));
    p = f2_fma(p, t, f2_pack(0.5f * kAS_a1, 0.5f * kAS_a1));
    p = f2_mul(p, t);
    const float ce = -0.72134752044448170f;  // -log2(e) / 2
    float w0, w1;
    f2_unpack(f2_mul(f2_mul(z, z), f2_pack(ce, ce)), w0, w1);
    const unsigned long long e = f2_pack(ex2_approx(w0), ex2_approx(w1));
    const unsigned long long half = f2_pack(0.5f, 0.5f);
    f2_unpack(f2_fma(az, f2_sub(half, f2_mul(p, e)), f2_mul(half, z)), g0, g1);
}
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---------------------------------------------------------------- GEMM
// C[M x N] = A[M x K] . B[N x K]^T, A and B row-major BF16 (K contiguous).
// Rows of A at or beyond m_valid and rows of B at or beyond n_valid read as 0.
struct Gemm {
    const __nv_bfloat16 *A;
    int lda, m_valid;
    const __nv_bfloat16 *B;
    int ldb, n_valid;
    int M, N, K;
    float *C;               // mode 0: FP32 store of rows < m_valid, cols < n_valid
    int ldc;
    const float *bias;      // mode 1: z = acc + bias
    float *Z;               // mode 1: pre-activation (optional), [M][N]
    __nv_bfloat16 *H, *HT;  // mode 1: gelu(z) as [M][N] and (optional) [N][ldt]
    const float *Zin;       // mode 2: dz = acc * gelu'(Zin)
    __nv_bfloat16 *dZ, *dZT;
    float *db;              // mode 2: column sums of dz (atomic)
    int ldt;
    int *err;
};

template <int MODE>
__global__ void __launch_bounds__(128, 1) umma_gemm(Gemm g) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    uint8_t *sA = smem;
    uint8_t *sB = smem + kTileM * kKC * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileM;
    const int KC = g.K < kKC ? g.K : kKC;
    const int cpr = KC / 8;  // 16-byte chunks per row of a K chunk
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = mma_idesc(kTileM, g.N);
    uint32_t phase = 0;
    int ok = 1;
    for (int k0 = 0; k0 < g.K; k0 += KC) {
        // stage the K chunk: core matrix (i, j) of 8 rows x 8 elements at
        // i * (cpr * 128) + j * 128 bytes, row r of it at 16 r
        for (int c = tid; c < kTileM * cpr; c += 128) {
            const int r = c / cpr, j = c % cpr, gr = m0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (gr < g.m_valid) v = *reinterpret_cast<const uint4 *>(g.A + (size_t)gr * g.lda + k0 + 8 * j);
            *reinterpret_cast<uint4 *>(sA + (r >> 3) * (cpr * 128) + j * 128 + (r & 7) * 16) = v;
        }
        for (int c = tid; c < g.N * cpr; c += 128) {
            const int r = c / cpr, j = c % cpr;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r < g.n_valid) v = *reinterpret_cast<const uint4 *>(g.B + (size_t)r * g.ldb + k0 + 8 * j);
            *reinterpret_cast<uint4 *>(sB + (r >> 3) * (cpr * 128) + j * 128 + (r & 7) * 16) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async proxy
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int s = 0; s < KC / 16; ++s) {
                const uint64_t ad = smem_desc(smem_addr(sA + s * 256), 128, cpr * 128);
                const uint64_t bd = smem_desc(smem_addr(sB + s * 256), 128, cpr * 128);
                mma_bf16(tmem, ad, bd, idesc, (k0 > 0 || s > 0) ? 1 : 0);
            }
            mma_commit(&mbar);
        }
        // the tile may be overwritten only after the products that read it finished
        const int done = mbar_wait(&mbar, phase) ? 1 : 0;
        ok = __syncthreads_and(done);
        phase ^= 1;
        if (!ok) break;
    }
    if (!ok) {
        // record, then give products still in flight a bounded second chance
        if (tid == 0) atomicExch(g.err, 1);
        mbar_wait(&mbar, phase ^ 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int m = m0 + warp * 32 + lane;
        for (int cb = 0; cb < g.N / 16; ++cb) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16), v);
            float gv[16];
            if (MODE == 1) {
#pragma unroll
                for (int e = 0; e < 16; e += 2)
                    gelu2(__fadd_rn(v[e], g.bias[cb * 16 + e]), __fadd_rn(v[e + 1], g.bias[cb * 16 + e + 1]), gv[e],
                          gv[e + 1]);
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int n = cb * 16 + e;
                if (MODE == 0) {
                    if (m < g.m_valid && n < g.n_valid) g.C[(size_t)m * g.ldc + n] = v[e];
                } else if (MODE == 1) {
                    const float z = __fadd_rn(v[e], g.bias[n]);
                    if (g.Z) g.Z[(size_t)m * g.N + n] = z;
                    const __nv_bfloat16 h = __float2bfloat16_rn(gv[e]);
                    g.H[(size_t)m * g.N + n] = h;
                    if (g.HT) g.HT[(size_t)n * g.ldt + m] = h;
                } else {
                    const float dz = v[e] * gelu_grad(g.Zin[(size_t)m * g.N + n]);
                    const __nv_bfloat16 d = __float2bfloat16_rn(dz);
                    g.dZ[(size_t)m * g.N + n] = d;
                    g.dZT[(size_t)n * g.ldt + m] = d;
                    float s = __bfloat162float(d);
#pragma unroll
                    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) atomicAdd(g.db + n, s);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ---------------------------------------------------------------- fused forward
// Inference in one persistent kernel.  A CTA takes 128-row tiles in turn and
// keeps everything between the inputs and the output on the chip: the
// activation of the current layer is the A operand in shared memory (128 x 256
// BF16 in the canonical K-major layout, core matrix (i, j) at i * 4096 + j * 128),
// the accumulator lives in tensor memory, and the weights stream from L2
// through a ring of 8 KB slots in the order the products consume them: W1
// (256 x 16) in one slot, W2 and W3 as sixteen K = 16 slices of 256 rows each,
// and the 16-row padded W4 (all sixteen K steps, 512 bytes apiece) in one slot.
// Warp 8 issues the bulk copies, one lane of warp 9 the products, warps 0-7
// the epilogues (two warps per quarter of the TMEM lanes, one per column
// half); the epilogue warps hand each A operand to the product lane through
// an mbarrier, and every wait is bounded (WLB_ERR_TIMEOUT, then the kernel
// drains its copies and products and frees the tensor memory).
// Products, epilogue arithmetic and BF16 roundings are those of the
// layer-by-layer path, so the two give the same bits.
constexpr int kSlots = 5, kSlotBytes = 8192, kChunks = 34;
constexpr int kActBytes = kTileM * kHid * 2;
constexpr int kFusedSmem = kActBytes + kSlots * kSlotBytes + 1024;
constexpr int kEpiThreads = 256, kProducerWarp = 8, kMmaWarp = 9, kFusedThreads = 320;

struct Fused {
    const float *x;
    long long n;
    float *y;
    unsigned char *inside;   // optional
    const float *lo, *hi;
    const float *w;          // FP32 masters: biases at ob1, ob2, ob3, ob4
    const uint8_t *stream;   // kChunks x kSlotBytes, written by pack_stream
    long long tiles;
    int *err;
};

__device__ __forceinline__ void mbar_expect(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(mbar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}

// Bounded wait that also gives up once another role has raised `abort`.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *mbar, uint32_t phase, volatile int *abort) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        if (mbar_try(mbar, phase)) return true;
        if ((i & 255) == 255 && *abort) return false;
    }
    return false;
}


__global__ void __launch_bounds__(kFusedThreads, 2) mlp_forward_fused(Fused a) {
    extern __shared__ uint8_t fused_raw[];
    uint8_t *act = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(fused_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *ring = act + kActBytes;
    __shared__ float s_bias[3][kHid];
    __shared__ uint64_t full[kSlots], empty[kSlots], accum, act_ready, drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort_store;
    volatile int *s_abort = &s_abort_store;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long my_tiles = blockIdx.x < a.tiles ? (a.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    for (int i = tid; i < 3 * kHid; i += kFusedThreads) {
        const int l = i / kHid;
        s_bias[l][i % kHid] = a.w[(l == 0 ? ob1 : l == 1 ? ob2 : ob3) + i % kHid];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty[s])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&accum)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&act_ready)), "r"(kEpiThreads));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&drain)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == kProducerWarp) {
        // the weight slices of every tile, in consumption order
        if (lane == 0) {
            const uint8_t *src = a.stream;
            const long long total = my_tiles * kChunks;
            // 32-bit counters advanced by increment: the loop is on the critical path
            int slot = 0, chunk = 0;
            uint32_t round_par = 0;  // parity of c / kSlots
            long long c = 0;
            for (; c < total; ++c) {
                if (c >= kSlots && !mbar_wait_or_abort(&empty[slot], round_par ^ 1u, s_abort)) {
                    if (!*s_abort) {
                        *s_abort = 1;
                        atomicExch(a.err, 1);
                    }
                    break;
                }
                mbar_expect(&full[slot], kSlotBytes);
                bulk_load(ring + slot * kSlotBytes, src + chunk * kSlotBytes, kSlotBytes, &full[slot]);
                if (++chunk == kChunks) chunk = 0;
                if (++slot == kSlots) {
                    slot = 0;
                    round_par ^= 1u;
                }
            }
            if (c < total) {
                // stopped early: the copies already issued land before the CTA exits
                for (int slot = 0; slot < kSlots; ++slot) {
                    const long long k = c > slot ? (c - slot + kSlots - 1) / kSlots : 0;
                    if (k > 0) mbar_wait(&full[slot], (uint32_t)((k - 1) & 1));
                }
            }
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // products: per layer, once the epilogue warps have written its A operand
        if (lane == 0) {
            const uint32_t id_hid = mma_idesc(kTileM, kHid), id_out = mma_idesc(kTileM, kOutPad);
            // descriptors: the start-address field (bits 0-13, address / 16) takes
            // the offsets directly (every address is below 256 KB)
            const uint64_t a_desc = smem_desc(smem_addr(act), 128, 4096);
            const uint64_t b_desc = smem_desc(smem_addr(ring), 128, 256);
            int slot = 0;
            uint32_t full_par = 0;  // parity of c / kSlots
            uint32_t ready_phase = 0;
            bool ok = true;
            for (long long t = 0; t < my_tiles && ok; ++t) {
                for (int layer = 0; layer < 4 && ok; ++layer) {
                    ok = mbar_wait_or_abort(&act_ready, ready_phase, s_abort);
                    ready_phase ^= 1;
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int slices = layer == 0 || layer == 3 ? 1 : kHid / 16;
                    for (int s = 0; s < slices; ++s) {
                        if (!mbar_wait_or_abort(&full[slot], full_par, s_abort)) {
                            ok = false;
                            break;
                        }
                        const uint64_t b = b_desc + (uint64_t)(slot * (kSlotBytes >> 4));
                        if (layer < 3) {
                            mma_bf16(tmem, a_desc + (uint64_t)(s * (256 >> 4)), b, id_hid, s > 0 ? 1 : 0);
                        } else {
                            for (int k = 0; k < kHid / 16; ++k)
                                mma_bf16(tmem, a_desc + (uint64_t)(k * (256 >> 4)), b + (uint64_t)(k * (512 >> 4)),
                                         id_out, k > 0 ? 1 : 0);
                        }
                        mma_commit(&empty[slot]);
                        if (++slot == kSlots) {
                            slot = 0;
                            full_par ^= 1u;
                        }
                    }
                    if (ok) mma_commit(&accum);
                }
            }
            if (!ok && !*s_abort) {
                *s_abort = 1;
                atomicExch(a.err, 1);
            }
            // no product may still be running when the tensor memory is freed
            mma_commit(&drain);
            mbar_wait(&drain, 0);
        }
        __syncwarp();
    } else {
        // epilogue warps: two per quarter of the TMEM lanes, one per column half
        const int q = warp & 3, col0 = (warp >> 2) * (kHid / 2);
        const int row = 32 * q + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        const float b4 = a.w[ob4];
        uint32_t acc_phase = 0;
        bool ok = true;
        for (long long t = 0; t < my_tiles && ok; ++t) {
            const long long m0 = (blockIdx.x + t * (long long)gridDim.x) * kTileM;
            {
                // normalised inputs: K = 16 columns, 4 of them real
                const int r = tid & (kTileM - 1), j = tid >> 7;
                uint32_t pk[4] = {0, 0, 0, 0};
                if (j == 0 && m0 + r < a.n) {
                    const float *xr = a.x + (m0 + r) * kIn;
                    for (int e = 0; e < kIn; e += 2) {
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(normalise_input(xr[e], a.lo[e], a.hi[e]));
                        const __nv_bfloat16 h1 =
                            __float2bfloat16_rn(normalise_input(xr[e + 1], a.lo[e + 1], a.hi[e + 1]));
                        pk[e / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    }
                }
                *reinterpret_cast<uint4 *>(act + (r >> 3) * 4096 + j * 128 + (r & 7) * 16) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&act_ready);
            for (int layer = 0; layer < 4; ++layer) {
                ok = mbar_wait_or_abort(&accum, acc_phase, s_abort);
                acc_phase ^= 1;
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (layer < 3) {
                    // bias + GELU -> BF16 -> the next layer's A operand
                    const float *bias = s_bias[layer];
                    // each column block's TMEM load is issued before the previous block's
                    // arithmetic, so its latency overlaps it
                    uint32_t rbuf[2][32];
                    tmem_ld32_issue(trow + (uint32_t)col0, rbuf[0]);
                    tmem_ld_wait(rbuf[0]);
#pragma unroll
                    for (int cb = 0; cb < kHid / 2 / 32; ++cb) {
                        const int n0 = col0 + 32 * cb;
                        if (cb + 1 < kHid / 2 / 32) tmem_ld32_issue(trow + (uint32_t)(n0 + 32), rbuf[(cb + 1) & 1]);
                        const uint32_t (&r)[32] = rbuf[cb & 1];
                        uint32_t pk[16];
#pragma unroll
                        for (int e = 0; e < 32; e += 2) {
                            float g0, g1;
                            gelu2(__fadd_rn(__uint_as_float(r[e]), bias[n0 + e]),
                                  __fadd_rn(__uint_as_float(r[e + 1]), bias[n0 + e + 1]), g0, g1);
                            const __nv_bfloat162 h = __floats2bfloat162_rn(g0, g1);
                            pk[e / 2] = *reinterpret_cast<const uint32_t *>(&h);
                        }
                        uint8_t *dst = act + (row >> 3) * 4096 + (n0 >> 3) * 128 + (row & 7) * 16;
#pragma unroll
                        for (int g = 0; g < 4; ++g)
                            *reinterpret_cast<uint4 *>(dst + 128 * g) =
                                make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
                        if (cb + 1 < kHid / 2 / 32) tmem_ld_wait(rbuf[(cb + 1) & 1]);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(&act_ready);
                } else if (col0 == 0) {
                    float v[16];
                    tmem_ld16(trow, v);
                    const long long i = m0 + row;
                    if (i < a.n) {
                        a.y[i] = v[0] + b4;
                        if (a.inside) {
                            bool in = true;
                            for (int e = 0; e < kIn; ++e) {
                                const float xv = a.x[i * kIn + e];
                                in &= xv >= a.lo[e] && xv <= a.hi[e];
                            }
                            a.inside[i] = in ? 1 : 0;
                        }
                    }
                }
            }
        }
        if (!ok && !*s_abort) {
            *s_abort = 1;
            atomicExch(a.err, 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// The weight stream of the fused forward (BF16, layout as described above).
__global__ void pack_stream(const float *__restrict__ w, __nv_bfloat16 *__restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int per = kSlotBytes / 2;
    if (e >= kChunks * per) return;
    const int c = e / per, ob = 2 * (e % per);
    float v = 0.0f;
    if (c < kChunks - 1) {
        // element (n, k) of a 256 x 16 slice at (n/8) 256 + (k/8) 128 + (n%8) 16 + (k%8) 2
        const int n = 8 * (ob / 256) + (ob % 128) / 16, k = 8 * ((ob % 256) / 128) + (ob % 16) / 2;
        if (c == 0)
            v = k < kIn ? w[oW1 + n * kIn + k] : 0.0f;
        else
            v = w[(c <= 16 ? oW2 : oW3) + n * kHid + 16 * ((c - 1) % 16) + k];
    } else {
        // W4 padded to 16 rows, K step s at 512 s
        const int r = 8 * ((ob % 512) / 256) + (ob % 128) / 16;
        const int k = 16 * (ob / 512) + 8 * ((ob % 256) / 128) + (ob % 16) / 2;
        v = r == 0 ? w[oW4 + k] : 0.0f;
    }
    out[e] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------- small kernels
// Inputs x (n x 4 FP32, optionally gathered through perm) -> normalised to
// [-1, 1] by the box [lo, hi], BF16 [B][16] and [16][B] (padding zero).
__global__ void prep_inputs(const float *__restrict__ x, const float *__restrict__ t, const int *__restrict__ perm,
                            long long first, int n, int Bp, const float *lo, const float *hi,
                            __nv_bfloat16 *__restrict__ X0, __nv_bfloat16 *__restrict__ X0T, float *__restrict__ tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp) return;
    const long long src = perm ? perm[first + i] : first + i;
    for (int a = 0; a < kInPad; ++a) {
        float v = 0.0f;
        if (i < n && a < kIn) v = normalise_input(x[src * kIn + a], lo[a], hi[a]);
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        X0[(size_t)i * kInPad + a] = h;
        X0T[(size_t)a * Bp + i] = h;
    }
    if (tb) tb[i] = (i < n && t) ? t[src] : 0.0f;
}

// MSE head: y = Y[:,0] + b4; loss += (y - t)^2 / n; dL/dy = 2 (y - t) / n.
__global__ void loss_head(const float *__restrict__ Y, const float *__restrict__ b4, const float *__restrict__ t,
                          int n, int Bp, __nv_bfloat16 *__restrict__ dZ4, __nv_bfloat16 *__restrict__ dZ4T,
                          float *__restrict__ db4, float *__restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp) return;
    float g = 0.0f, l = 0.0f;
    if (i < n) {
        const float d = Y[(size_t)i * kOutPad] + b4[0] - t[i];
        l = d * d / (float)n;
        g = 2.0f * d / (float)n;
    }
    const __nv_bfloat16 gb = __float2bfloat16_rn(g);
    for (int a = 0; a < kOutPad; ++a) {
        dZ4[(size_t)i * kOutPad + a] = a == 0 ? gb : __float2bfloat16_rn(0.0f);
        dZ4T[(size_t)a * Bp + i] = a == 0 ? gb : __float2bfloat16_rn(0.0f);
    }
    float s = __bfloat162float(gb);
    for (int o = 16; o >= 1; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        l += __shfl_xor_sync(0xffffffffu, l, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(db4, s);
        atomicAdd(loss, l);
    }
}

__global__ void predict_head(const float *__restrict__ Y, const float *__restrict__ b4, const float *__restrict__ x,
                             long long first, int n, const float *lo, const float *hi, float *__restrict__ y,
                             unsigned char *__restrict__ inside) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[first + i] = Y[(size_t)i * kOutPad] + b4[0];
    if (inside) {
        bool in = true;
        for (int a = 0; a < kIn; ++a) {
            const float v = x[(first + i) * kIn + a];
            in &= v >= lo[a] && v <= hi[a];
        }
        inside[first + i] = in ? 1 : 0;
    }
}

// Adam on the FP32 masters (bias-corrected), then nothing else: BF16 copies
// are refreshed by pack_weights.
__global__ void adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                     float *__restrict__ m2, int n, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = 0.9f * m1[i] + 0.1f * gi;
    const float b = 0.999f * m2[i] + 0.001f * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * (a * c1) / (sqrtf(b * c2) + 1e-8f);
}

// BF16 working copies: W1 [256][16], W2, W3 [256][256], W4 [16][256] (padding
// zero) and the transposes W2^T, W3^T [256][256], W4^T [256][16].
__global__ void pack_weights(const float *__restrict__ w, __nv_bfloat16 *W1, __nv_bfloat16 *W2, __nv_bfloat16 *W3,
                             __nv_bfloat16 *W4, __nv_bfloat16 *W2T, __nv_bfloat16 *W3T, __nv_bfloat16 *W4T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 256 x 256
    if (i >= kHid * kHid) return;
    const int r = i / kHid, c = i % kHid;
    W2[i] = __float2bfloat16_rn(w[oW2 + i]);
    W3[i] = __float2bfloat16_rn(w[oW3 + i]);
    W2T[c * kHid + r] = __float2bfloat16_rn(w[oW2 + i]);
    W3T[c * kHid + r] = __float2bfloat16_rn(w[oW3 + i]);
    if (c < kInPad) W1[r * kInPad + c] = __float2bfloat16_rn(c < kIn ? w[oW1 + r * kIn + c] : 0.0f);
    if (r < kOutPad) {
        const __nv_bfloat16 v = __float2bfloat16_rn(r == 0 ? w[oW4 + c] : 0.0f);
        W4[r * kHid + c] = v;
        W4T[c * kOutPad + r] = v;
    }
}

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct wlb_mlp {
    int batch_max = 0;  // multiple of 128
    int device = 0;
    cudaStream_t stream = nullptr;
    void *mem = nullptr;
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    float *lo = nullptr, *hi = nullptr, *loss = nullptr, *tb = nullptr;
    __nv_bfloat16 *W1, *W2, *W3, *W4, *W2T, *W3T, *W4T;
    __nv_bfloat16 *X0, *X0T, *H[3], *HT[3], *dZ[3], *dZT[3], *dZ4, *dZ4T;
    float *Z[3], *Y;
    uint8_t *Wstream = nullptr;  // fused-forward weight stream (kChunks x kSlotBytes)
    bool stream_stale = true;    // weights changed since the stream was packed
    bool fused = true;           // predict through mlp_forward_fused
    int fused_grid = 0;          // CTAs of the fused forward (SMs x resident CTAs)
    int *err = nullptr, *perm = nullptr;
    long long perm_cap = 0;
    float host_lo[4], host_hi[4];
    long long adam_t = 0;
    char msg[512] = {0};
};

namespace {

wlb_status mfail(wlb_mlp *m, wlb_status s, const char *what, cudaError_t e = cudaSuccess) {
    if (m) snprintf(m->msg, sizeof(m->msg), "%s%s%s", what, e != cudaSuccess ? ": " : "",
                    e != cudaSuccess ? cudaGetErrorString(e) : "");
    return s;
}

#define MLP_CUDA(m, call, what)                                           \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return mfail((m), WLB_ERR_CUDA, (what), e_); \
    } while (0)

template <int MODE>
cudaError_t run_gemm(const Gemm &g, cudaStream_t s) {
    static bool configured = false;  // per process; attribute applies to the current device
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(umma_gemm<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    umma_gemm<MODE><<<g.M / kTileM, 128, kSmemBytes, s>>>(g);
    return cudaGetLastError();
}

Gemm base_gemm(wlb_mlp *m) {
    Gemm g{};
    g.err = m->err;
    return g;
}

// Forward of one padded batch of Bp rows (X0 staged).  keep: store Z and H^T.
cudaError_t forward(wlb_mlp *m, int Bp, bool keep) {
    const __nv_bfloat16 *Win[3] = {m->W1, m->W2, m->W3};
    const int Kin[3] = {kInPad, kHid, kHid};
    const float *bias[3] = {m->w + ob1, m->w + ob2, m->w + ob3};
    const __nv_bfloat16 *A = m->X0;
    for (int l = 0; l < 3; ++l) {
        Gemm g = base_gemm(m);
        g.A = A; g.lda = Kin[l]; g.m_valid = Bp;
        g.B = Win[l]; g.ldb = Kin[l]; g.n_valid = kHid;
        g.M = Bp; g.N = kHid; g.K = Kin[l];
        g.bias = bias[l];
        g.Z = keep ? m->Z[l] : nullptr;
        g.H = m->H[l];
        g.HT = keep ? m->HT[l] : nullptr;
        g.ldt = Bp;
        cudaError_t e = run_gemm<1>(g, m->stream);
        if (e != cudaSuccess) return e;
        A = m->H[l];
    }
    Gemm g = base_gemm(m);
    g.A = m->H[2]; g.lda = kHid; g.m_valid = Bp;
    g.B = m->W4; g.ldb = kHid; g.n_valid = kOutPad;
    g.M = Bp; g.N = kOutPad; g.K = kHid;
    g.C = m->Y; g.ldc = kOutPad;
    return run_gemm<0>(g, m->stream);
}

// Loss and gradients of one staged batch (n real rows of Bp) into m->g.
cudaError_t backward(wlb_mlp *m, int n, int Bp) {
    cudaError_t e = cudaMemsetAsync(m->g, 0, sizeof(float) * kParams, m->stream);
    if (e != cudaSuccess) return e;
    if ((e = forward(m, Bp, true)) != cudaSuccess) return e;
    loss_head<<<(Bp + 127) / 128, 128, 0, m->stream>>>(m->Y, m->w + ob4, m->tb, n, Bp, m->dZ4, m->dZ4T, m->g + ob4,
                                                        m->loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // layer 4: dW4 = dZ4^T H3, dH3 = dZ4 W4 -> dZ3
    const __nv_bfloat16 *dA = m->dZ4, *dAT = m->dZ4T;
    int kprev = kOutPad, mrows = 1;
    const __nv_bfloat16 *WT[3] = {m->W2T, m->W3T, m->W4T};  // W_{l+1}^T for l = 0..2
    const int gW[4] = {oW1, oW2, oW3, oW4};
    const int gb[3] = {ob1, ob2, ob3};
    for (int l = 2; l >= 0; --l) {
        // weight gradient of layer l+2 (1-based): dW = dA^T . H_l
        Gemm w = base_gemm(m);
        w.A = dAT; w.lda = Bp; w.m_valid = mrows;
        w.B = m->HT[l]; w.ldb = Bp; w.n_valid = kHid;
        w.M = ((mrows + kTileM - 1) / kTileM) * kTileM; w.N = kHid; w.K = Bp;
        w.C = m->g + gW[l + 1]; w.ldc = kHid;
        if ((e = run_gemm<0>(w, m->stream)) != cudaSuccess) return e;
        // activation gradient: dH_l = dA . W_{l+2}, dZ_l = dH_l * gelu'(Z_l)
        Gemm d = base_gemm(m);
        d.A = dA; d.lda = kprev; d.m_valid = Bp;
        d.B = WT[l]; d.ldb = kprev; d.n_valid = kHid;
        d.M = Bp; d.N = kHid; d.K = kprev;
        d.Zin = m->Z[l]; d.dZ = m->dZ[l]; d.dZT = m->dZT[l]; d.db = m->g + gb[l]; d.ldt = Bp;
        if ((e = run_gemm<2>(d, m->stream)) != cudaSuccess) return e;
        dA = m->dZ[l];
        dAT = m->dZT[l];
        kprev = kHid;
        mrows = kHid;
    }
    // layer 1: dW1 = dZ1^T . X0 (4 real input columns)
    Gemm w = base_gemm(m);
    w.A = m->dZT[0]; w.lda = Bp; w.m_valid = kHid;
    w.B = m->X0T; w.ldb = Bp; w.n_valid = kIn;
    w.M = kHid; w.N = kInPad; w.K = Bp;
    w.C = m->g + oW1; w.ldc = kIn;
    return run_gemm<0>(w, m->stream);
}

cudaError_t stage(wlb_mlp *m, const float *x, const float *t, const int *perm, long long first, int n, int Bp) {
    prep_inputs<<<(Bp + 127) / 128, 128, 0, m->stream>>>(x, t, perm, first, n, Bp, m->lo, m->hi, m->X0, m->X0T,
                                                          m->tb);
    return cudaGetLastError();
}

cudaError_t repack(wlb_mlp *m) {
    m->stream_stale = true;
    pack_weights<<<(kHid * kHid + 255) / 256, 256, 0, m->stream>>>(m->w, m->W1, m->W2, m->W3, m->W4, m->W2T,
                                                                   m->W3T, m->W4T);
    return cudaGetLastError();
}

// Whole inference in one launch of the fused kernel (n >= 1).
cudaError_t forward_fused(wlb_mlp *m, const float *x, long long n, float *y, unsigned char *inside) {
    cudaError_t e;
    if (m->stream_stale) {
        pack_stream<<<(kChunks * kSlotBytes / 2 + 255) / 256, 256, 0, m->stream>>>(
            m->w, reinterpret_cast<__nv_bfloat16 *>(m->Wstream));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        m->stream_stale = false;
    }
    if (m->fused_grid == 0) {
        // the attribute applies to the current device, set for every handle
        if ((e = cudaFuncSetAttribute(mlp_forward_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kFusedSmem)) != cudaSuccess)
            return e;
        // two CTAs per SM need the largest shared-memory carveout
        if ((e = cudaFuncSetAttribute(mlp_forward_fused, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
            return e;
        // resident CTAs per SM from the SM's shared memory and registers, at
        // most two (each holds half of the tensor memory)
        int sms = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
        cudaFuncAttributes fa{};
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, m->device)) !=
                cudaSuccess ||
            (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, m->device)) !=
                cudaSuccess ||
            (e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, m->device)) !=
                cudaSuccess ||
            (e = cudaFuncGetAttributes(&fa, mlp_forward_fused)) != cudaSuccess)
            return e;
        const long long smem_block = (long long)fa.sharedSizeBytes + kFusedSmem + reserved;
        const long long regs_block = (long long)fa.numRegs * kFusedThreads;
        long long per_sm = 2;
        if (smem_sm / smem_block < per_sm) per_sm = smem_sm / smem_block;
        if (regs_block > 0 && regs_sm / regs_block < per_sm) per_sm = regs_sm / regs_block;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        m->fused_grid = (int)(sms * per_sm);
    }
    Fused f{};
    f.x = x; f.n = n; f.y = y; f.inside = inside;
    f.lo = m->lo; f.hi = m->hi; f.w = m->w;
    f.stream = m->Wstream;
    f.tiles = (n + kTileM - 1) / kTileM;
    f.err = m->err;
    const long long grid = f.tiles < m->fused_grid ? f.tiles : m->fused_grid;
    mlp_forward_fused<<<(unsigned)grid, kFusedThreads, kFusedSmem, m->stream>>>(f);
    return cudaGetLastError();
}

wlb_status check_err(wlb_mlp *m) {
    int flag = 0;
    MLP_CUDA(m, cudaMemcpyAsync(&flag, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream), "flag copy");
    MLP_CUDA(m, cudaStreamSynchronize(m->stream), "synchronize");
    if (flag) return mfail(m, WLB_ERR_TIMEOUT, "tensor-core wait limit reached");
    return WLB_OK;
}

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int wlb_mlp_param_count(void) { return kParams; }

wlb_status wlb_mlp_create(int batch_max, const float x_lo[4], const float x_hi[4], void *stream, wlb_mlp **out) {
    if (!out || !x_lo || !x_hi || batch_max < 128 || batch_max % 128 != 0 || batch_max > (1 << 22))
        return WLB_ERR_ARG;
    for (int a = 0; a < 4; ++a)
        if (!(x_hi[a] > x_lo[a])) return WLB_ERR_ARG;
    wlb_mlp *m = new (std::nothrow) wlb_mlp();
    if (!m) return WLB_ERR_OOM;
    m->batch_max = batch_max;
    m->stream = (cudaStream_t)stream;
    memcpy(m->host_lo, x_lo, sizeof(m->host_lo));
    memcpy(m->host_hi, x_hi, sizeof(m->host_hi));
    const size_t B = (size_t)batch_max, H = kHid;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += a256(bytes); return o; };
    const size_t ow = take(4 * kParams), og = take(4 * kParams), om1 = take(4 * kParams), om2 = take(4 * kParams);
    const size_t olo = take(16), ohi = take(16), oloss = take(4), otb = take(4 * B), oerr = take(4);
    const size_t oW1 = take(2 * H * kInPad), oW2 = take(2 * H * H), oW3 = take(2 * H * H), oW4 = take(2 * kOutPad * H);
    const size_t oW2T = take(2 * H * H), oW3T = take(2 * H * H), oW4T = take(2 * H * kOutPad);
    const size_t oX0 = take(2 * B * kInPad), oX0T = take(2 * B * kInPad);
    size_t oH[3], oHT[3], odZ[3], odZT[3], oZ[3];
    for (int l = 0; l < 3; ++l) {
        oH[l] = take(2 * B * H); oHT[l] = take(2 * B * H); odZ[l] = take(2 * B * H); odZT[l] = take(2 * B * H);
        oZ[l] = take(4 * B * H);
    }
    const size_t odZ4 = take(2 * B * kOutPad), odZ4T = take(2 * B * kOutPad), oY = take(4 * B * kOutPad);
    const size_t oWs = take((size_t)kChunks * kSlotBytes);
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaMalloc(&m->mem, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return WLB_ERR_OOM;
    }
    char *p = (char *)m->mem;
    m->w = (float *)(p + ow); m->g = (float *)(p + og); m->m1 = (float *)(p + om1); m->m2 = (float *)(p + om2);
    m->lo = (float *)(p + olo); m->hi = (float *)(p + ohi); m->loss = (float *)(p + oloss); m->tb = (float *)(p + otb);
    m->err = (int *)(p + oerr);
    m->W1 = (__nv_bfloat16 *)(p + oW1); m->W2 = (__nv_bfloat16 *)(p + oW2); m->W3 = (__nv_bfloat16 *)(p + oW3);
    m->W4 = (__nv_bfloat16 *)(p + oW4); m->W2T = (__nv_bfloat16 *)(p + oW2T); m->W3T = (__nv_bfloat16 *)(p + oW3T);
    m->W4T = (__nv_bfloat16 *)(p + oW4T);
    m->X0 = (__nv_bfloat16 *)(p + oX0); m->X0T = (__nv_bfloat16 *)(p + oX0T);
    for (int l = 0; l < 3; ++l) {
        m->H[l] = (__nv_bfloat16 *)(p + oH[l]); m->HT[l] = (__nv_bfloat16 *)(p + oHT[l]);
        m->dZ[l] = (__nv_bfloat16 *)(p + odZ[l]); m->dZT[l] = (__nv_bfloat16 *)(p + odZT[l]);
        m->Z[l] = (float *)(p + oZ[l]);
    }
    m->dZ4 = (__nv_bfloat16 *)(p + odZ4); m->dZ4T = (__nv_bfloat16 *)(p + odZ4T); m->Y = (float *)(p + oY);
    m->Wstream = (uint8_t *)(p + oWs);
    e = cudaMemsetAsync(m->mem, 0, off, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->lo, x_lo, 16, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->hi, x_hi, 16, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        wlb_mlp_destroy(m);
        return WLB_ERR_CUDA;
    }
    *out = m;
    return WLB_OK;
}

wlb_status wlb_mlp_set_weights(wlb_mlp *m, const float *w) {
    if (!m || !w) return WLB_ERR_ARG;
    MLP_CUDA(m, cudaMemcpyAsync(m->w, w, sizeof(float) * kParams, cudaMemcpyHostToDevice, m->stream), "weights");
    MLP_CUDA(m, cudaMemsetAsync(m->m1, 0, sizeof(float) * kParams, m->stream), "adam state");
    MLP_CUDA(m, cudaMemsetAsync(m->m2, 0, sizeof(float) * kParams, m->stream), "adam state");
    m->adam_t = 0;
    MLP_CUDA(m, repack(m), "pack");
    MLP_CUDA(m, cudaStreamSynchronize(m->stream), "synchronize");
    return WLB_OK;
}

wlb_status wlb_mlp_init_weights(wlb_mlp *m, unsigned long long seed) {
    if (!m) return WLB_ERR_ARG;
    std::vector<float> w(kParams);
    uint64_t s = seed;
    const int fan[8] = {kIn, kIn, kHid, kHid, kHid, kHid, kHid, kHid};
    const int off[9] = {oW1, ob1, oW2, ob2, oW3, ob3, oW4, ob4, kParams};
    for (int k = 0; k < 8; ++k) {
        const float a = 1.0f / std::sqrt((float)fan[k]);
        for (int i = off[k]; i < off[k + 1]; ++i) {
            const double u = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
            w[i] = (float)((2.0 * u - 1.0) * a);
        }
    }
    return wlb_mlp_set_weights(m, w.data());
}

wlb_status wlb_mlp_get_weights(wlb_mlp *m, float *w) {
    if (!m || !w) return WLB_ERR_ARG;
    MLP_CUDA(m, cudaMemcpyAsync(w, m->w, sizeof(float) * kParams, cudaMemcpyDeviceToHost, m->stream), "weights");
    MLP_CUDA(m, cudaStreamSynchronize(m->stream), "synchronize");
    return WLB_OK;
}

wlb_status wlb_mlp_loss_grad(wlb_mlp *m, const float *x, const float *t, int n, float *loss, float *grad) {
    if (!m || !x || !t || n < 1 || n > m->batch_max) return WLB_ERR_ARG;
    const int Bp = ((n + kTileM - 1) / kTileM) * kTileM;
    MLP_CUDA(m, cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream), "zero loss");
    MLP_CUDA(m, stage(m, x, t, nullptr, 0, n, Bp), "stage");
    MLP_CUDA(m, backward(m, n, Bp), "backward");
    wlb_status s = check_err(m);
    if (s != WLB_OK) return s;
    if (loss) MLP_CUDA(m, cudaMemcpy(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost), "loss");
    if (grad) MLP_CUDA(m, cudaMemcpy(grad, m->g, sizeof(float) * kParams, cudaMemcpyDeviceToHost), "grad");
    return WLB_OK;
}

wlb_status wlb_mlp_train(wlb_mlp *m, const float *x, const float *t, long long n, int epochs, int batch, float lr,
                         float lr_final, unsigned long long seed, float *loss_history) {
    if (!m || !x || !t || n < 1 || epochs < 1 || batch < 128 || batch % 128 != 0 || batch > m->batch_max ||
        !(lr > 0) || !(lr_final > 0))
        return WLB_ERR_ARG;
    if (m->perm_cap < n) {
        if (m->perm) cudaFree(m->perm);
        m->perm = nullptr;
        MLP_CUDA(m, cudaMalloc(&m->perm, sizeof(int) * n), "permutation buffer");
        m->perm_cap = n;
    }
    std::vector<int> perm((size_t)n);
    uint64_t s = seed;
    const long long nb = n / batch;  // whole batches per epoch
    if (nb < 1) return WLB_ERR_ARG;
    for (int ep = 0; ep < epochs; ++ep) {
        for (long long i = 0; i < n; ++i) perm[(size_t)i] = (int)i;
        for (long long i = n - 1; i > 0; --i) {  // Fisher-Yates
            const long long j = (long long)(splitmix(s) % (uint64_t)(i + 1));
            const int tmp = perm[(size_t)i];
            perm[(size_t)i] = perm[(size_t)j];
            perm[(size_t)j] = tmp;
        }
        MLP_CUDA(m, cudaMemcpyAsync(m->perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, m->stream), "perm");
        MLP_CUDA(m, cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream), "zero loss");
        const float lr_e = lr * std::pow(lr_final / lr, (float)ep / (float)(epochs > 1 ? epochs - 1 : 1));
        for (long long k = 0; k < nb; ++k) {
            MLP_CUDA(m, stage(m, x, t, m->perm, k * batch, batch, batch), "stage");
            MLP_CUDA(m, backward(m, batch, batch), "backward");
            m->adam_t += 1;
            const float c1 = 1.0f / (1.0f - std::pow(0.9f, (float)m->adam_t));
            const float c2 = 1.0f / (1.0f - std::pow(0.999f, (float)m->adam_t));
            adam<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->w, m->g, m->m1, m->m2, kParams, lr_e, c1, c2);
            MLP_CUDA(m, cudaGetLastError(), "adam");
            MLP_CUDA(m, repack(m), "pack");
        }
        float l = 0;
        MLP_CUDA(m, cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream), "loss");
        wlb_status st = check_err(m);
        if (st != WLB_OK) return st;
        if (loss_history) loss_history[ep] = l / (float)nb;
    }
    return WLB_OK;
}

wlb_status wlb_mlp_predict(wlb_mlp *m, const float *x, long long n, float *y, unsigned char *inside) {
    if (!m || n < 0 || (n > 0 && (!x || !y))) return WLB_ERR_ARG;
    if (m->fused) {
        if (n > 0) MLP_CUDA(m, forward_fused(m, x, n, y, inside), "fused forward");
        return check_err(m);
    }
    for (long long first = 0; first < n; first += m->batch_max) {
        const int cnt = (int)((n - first) < m->batch_max ? (n - first) : m->batch_max);
        const int Bp = ((cnt + kTileM - 1) / kTileM) * kTileM;
        MLP_CUDA(m, stage(m, x, nullptr, nullptr, first, cnt, Bp), "stage");
        MLP_CUDA(m, forward(m, Bp, false), "forward");
        predict_head<<<(cnt + 255) / 256, 256, 0, m->stream>>>(m->Y, m->w + ob4, x, first, cnt, m->lo, m->hi, y,
                                                               inside);
        MLP_CUDA(m, cudaGetLastError(), "predict head");
    }
    return check_err(m);
}

wlb_status wlb_mlp_set_fused(wlb_mlp *m, int fused) {
    if (!m || (fused != 0 && fused != 1)) return WLB_ERR_ARG;
    m->fused = fused == 1;
    return WLB_OK;
}

const char *wlb_mlp_last_error(const wlb_mlp *m) { return m ? m->msg : ""; }

wlb_status wlb_mlp_destroy(wlb_mlp *m) {
    if (!m) return WLB_ERR_ARG;
    if (m->perm) cudaFree(m->perm);
    if (m->mem) cudaFree(m->mem);
    delete m;
    return WLB_OK;
}

}  // extern "C"
