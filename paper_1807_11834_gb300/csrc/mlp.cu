// mlp.cu -- the learned drag closure (not in the paper): a small multilayer
// perceptron c = f(features) that scales the drag computed from stale bulk
// fields, trained and evaluated by this library's own tensor-core kernels.
//
// Network (features padded to 16 inputs, hidden width 64):
//   Z1 = X W1 + b1, A1 = act(Z1); Z2 = A1 W2 + b2, A2 = act(Z2); c = A2 w3 + b3
// act is GELU (the exact erf form) or ReLU, chosen per closure.  Weights are
// kept as FP32 master copies; the matrix products take BF16 operands with
// FP32 accumulation on the 5th generation tensor cores: a CTA of 128
// threads owns a tile of 128 rows, stages BF16 operands in shared memory in
// the no-swizzle K-major core-matrix layout, one thread issues tcgen05.mma
// into tensor memory (TMEM), completion is tracked by an mbarrier (bounded
// wait), and each thread reads back its row with tcgen05.ld.  The biases
// b1 and b2 ride in the products: three operand columns of ones meet the
// bias split into three BF16 terms whose sum is the FP32 bias exactly, so
// the epilogue between the products is the activation alone.  The small
// weight-gradient products (A^T dZ) run in FP32 on the CUDA cores in a
// fixed order, so training is deterministic.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>

#include <cuda_bf16.h>

#include "cg_internal.cuh"
#include "drag_law.cuh"

namespace cg {
namespace mlp {

constexpr int K0 = 16;                 // padded input width
constexpr int H = 64;                  // hidden width
constexpr int NFEAT = 7;               // used inputs
constexpr int KA = H + 16;             // K of the second product: 64 activations, 3 bias columns, zeros
constexpr int ACT_GELU = CG_MLP_GELU;
constexpr int ACT_RELU = CG_MLP_RELU;
constexpr int FEAT_STRIDE = 8;         // floats per feature row in memory
constexpr int OFF_W1 = 0;              // [K0][H]
constexpr int OFF_B1 = OFF_W1 + K0 * H;
constexpr int OFF_W2 = OFF_B1 + H;     // [H][H] (in, out)
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H;
constexpr int NPARAM = OFF_B3 + 1;     // 5313
constexpr int TILE = 128;              // rows per CTA tile
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr uint32_t kInferCols = 64;     // TMEM columns of a forward-only CTA (Z1, then Z2 in the same columns)
constexpr uint32_t kTrainCols = 256;    // Z1 (0..63), Z2 (64..127), dA1 (128..191)

// ---------------------------------------------------------------------------
// tcgen05 / TMEM / mbarrier primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Bounded wait for the given phase parity (at most `limit` polls); returns
// false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kSpinLimit) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(saddr(bar)), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// Shared-memory matrix descriptor: no swizzle, K-major core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups along M (or N).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture
    return d;                 // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 accumulate, both
// operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major core-matrix tile with K columns.
__host__ __device__ constexpr uint32_t koff(int row, int k, int K) {
    return (uint32_t)((row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// Two values as a BF16 pair (lo in the low half), rounded to nearest even;
// the relu form clamps negative results to zero in the same instruction.
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t bf16x2_relu(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Store 8 consecutive K values of one row (one 16-byte core-matrix row).
__device__ __forceinline__ void st_row8(unsigned char* tile, int row, int k0, int K, const float* v) {
    *reinterpret_cast<uint4*>(tile + koff(row, k0, K)) =
        make_uint4(bf16x2(v[0], v[1]), bf16x2(v[2], v[3]), bf16x2(v[4], v[5]), bf16x2(v[6], v[7]));
}

// Term j (0, 1, 2) of the split of an FP32 value into three BF16 values
// whose sum is the value exactly: h = bf16(b); the remainder b - h is exact
// in FP32 and holds at most 16 significant bits, m = bf16(b - h), and the
// last remainder b - h - m (exact again) fits the 8 bits of a BF16.
__device__ __forceinline__ float bias_term(float b, int j) {
    const float h = bf16_val(bf16_bits(b));
    if (j == 0) return h;
    const float r = b - h;
    const float m = bf16_val(bf16_bits(r));
    return j == 1 ? m : r - m;
}

// GELU x Phi(x) of the forward pass, with the complementary error function
// from formula 7.1.26 of Abramowitz & Stegun (Handbook of Mathematical
// Functions): erfc(z) ~ t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-z^2),
// t = 1 / (1 + p z), z >= 0, absolute error below 1.5e-7.  With
// q = erfc(|x| / sqrt 2) / 2: GELU(x) = x (1 - q) for x >= 0, x q otherwise.
__device__ __forceinline__ float gelu(float x) {
    const float z = fabsf(x) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, z, 1.0f));
    float p = fmaf(t, 1.061405429f, -1.453152027f);
    p = fmaf(t, p, 1.421413741f);
    p = fmaf(t, p, -0.284496736f);
    p = fmaf(t, p, 0.254829592f);
    const float q = 0.5f * t * p * __expf(-z * z);
    return x >= 0.f ? x - x * q : x * q;
}
// Two activations at once: the same formula with the FP32 arithmetic in
// packed f32x2 instructions (two lanes per instruction) and the reciprocal
// and the exponential on the special-function unit (rcp / ex2 approx).
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    return (unsigned long long)__float_as_uint(a) | ((unsigned long long)__float_as_uint(b) << 32);
}
__device__ __forceinline__ float lo2(unsigned long long v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float hi2(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void gelu2(float a, float b, float& ga, float& gb) {
    const unsigned long long z = mul2(pk2(fabsf(a), fabsf(b)), pk2(0.70710678118654752f, 0.70710678118654752f));
    const unsigned long long den = fma2(pk2(0.3275911f, 0.3275911f), z, pk2(1.0f, 1.0f));
    const unsigned long long t = pk2(rcp_approx(lo2(den)), rcp_approx(hi2(den)));
    unsigned long long p = fma2(t, pk2(1.061405429f, 1.061405429f), pk2(-1.453152027f, -1.453152027f));
    p = fma2(t, p, pk2(1.421413741f, 1.421413741f));
    p = fma2(t, p, pk2(-0.284496736f, -0.284496736f));
    p = fma2(t, p, pk2(0.254829592f, 0.254829592f));
    // exp(-z^2) = 2^(-z^2 log2 e)
    const unsigned long long zz = mul2(mul2(z, z), pk2(-1.4426950408889634f, -1.4426950408889634f));
    const unsigned long long e = pk2(ex2_approx(lo2(zz)), ex2_approx(hi2(zz)));
    const unsigned long long q = mul2(mul2(mul2(t, pk2(0.5f, 0.5f)), p), e);
    const unsigned long long xq = mul2(pk2(a, b), q);
    ga = a >= 0.f ? a - lo2(xq) : lo2(xq);
    gb = b >= 0.f ? b - hi2(xq) : hi2(xq);
}

// Its derivative Phi(x) + x phi(x) (training only), from CUDA's erff / expf.
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// ---------------------------------------------------------------------------
// Shared-memory layout of a CTA: the forward part, and the extra operands of
// the training kernel
// ---------------------------------------------------------------------------
// The network's forward operands as a CTA's shared memory holds them: built
// by k_mlp_image whenever the parameters change, copied by every CTA.
struct WeightImage {
    alignas(128) unsigned char W1t[H * K0 * 2];    // B of GEMM 1: (n = hidden, k = input; k 7..9: b1)
    alignas(128) unsigned char W2t[H * KA * 2];    // B of GEMM 2: (n = out, k = in; k 64..66: b2)
    float w3[H];
    float lo[FEAT_STRIDE], inv[FEAT_STRIDE];
    float b3;
};
static_assert(sizeof(WeightImage) % 16 == 0, "the image is copied in 16-byte words");
struct Smem {
    WeightImage w;
    alignas(128) unsigned char X[TILE * K0 * 2];   // A of GEMM 1 (columns 7..9: ones)
    alignas(128) unsigned char A1[TILE * KA * 2];  // A of GEMM 2 (BF16 act(Z1); columns 64..66: ones)
    uint64_t bar;
    uint32_t tmem;
    int fail;
};
struct SmemTrain {
    Smem s;
    alignas(128) unsigned char W2b[H * H * 2];     // B of the dA1 product: (n = in, k = out)
    alignas(128) unsigned char dZ2b[TILE * H * 2]; // A of the dA1 product (BF16 dZ2)
    float dZ2[TILE][H + 1];   // FP32 dZ2 (padded against bank conflicts)
    float dZ1[TILE][H + 1];   // FP32 dZ1
    float A2dc[TILE][H + 1];  // A2 * dc, for the w3 gradient
    float dc[TILE];
    float r2[TILE];
};

// The weight image from the FP32 parameters: BF16 operand copies of the
// weights with the split biases, and the FP32 vectors.  One CTA.
__global__ void __launch_bounds__(256)
k_mlp_image(const float* __restrict__ P, const float* __restrict__ scale, WeightImage* __restrict__ img) {
    for (int e = threadIdx.x; e < H * K0; e += blockDim.x) {
        const int n = e / K0, k = e % K0;   // W1t(n, k) = W1[k][n]; inputs past NFEAT are zero
        const float w = k < NFEAT ? P[OFF_W1 + k * H + n] : k < NFEAT + 3 ? bias_term(P[OFF_B1 + n], k - NFEAT) : 0.f;
        *reinterpret_cast<uint16_t*>(img->W1t + koff(n, k, K0)) = bf16_bits(w);
    }
    for (int e = threadIdx.x; e < H * KA; e += blockDim.x) {
        const int i = e / H, o = e % H;     // W2[i][o] as (n = out, k = in)
        const float w = i < H ? P[OFF_W2 + i * H + o] : i < H + 3 ? bias_term(P[OFF_B2 + o], i - H) : 0.f;
        *reinterpret_cast<uint16_t*>(img->W2t + koff(o, i, KA)) = bf16_bits(w);
    }
    for (int j = threadIdx.x; j < H; j += blockDim.x) img->w3[j] = P[OFF_W3 + j];
    if (threadIdx.x < FEAT_STRIDE) {
        img->lo[threadIdx.x] = scale[threadIdx.x];
        img->inv[threadIdx.x] = scale[FEAT_STRIDE + threadIdx.x];
    }
    if (threadIdx.x == 0) img->b3 = P[OFF_B3];
}

// A CTA's copy of the weight image (16-byte words, all in flight at once),
// and the constant columns of the second product's A tile (ones at
// 64..66, zeros up to KA), which no tile overwrites.
__device__ void load_weights(Smem& s, const WeightImage* __restrict__ img) {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    uint4* dst = reinterpret_cast<uint4*>(&s.w);
    constexpr int words = (int)(sizeof(WeightImage) / 16);
    for (int e = threadIdx.x; e < words; e += blockDim.x) dst[e] = __ldg(src + e);
    for (int row = threadIdx.x; row < TILE; row += blockDim.x) {
        const float one[8] = {1.f, 1.f, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f}, zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        st_row8(s.A1, row, H, KA, one);
        st_row8(s.A1, row, H + 8, KA, zero);
    }
}

// W2 as the B operand of dA1 = dZ2 W2^T (training).
__device__ void load_w2b(SmemTrain& st, const float* __restrict__ P) {
    for (int e = threadIdx.x; e < H * H; e += blockDim.x) {
        const int i = e / H, o = e % H;     // W2[i][o]
        *reinterpret_cast<uint16_t*>(st.W2b + koff(i, o, H)) = bf16_bits(P[OFF_W2 + i * H + o]);   // (n = in, k = out)
    }
}

// Scaled network input of one row from raw features (and the three ones
// that meet b1); returns in-range.
__device__ __forceinline__ bool scale_row(const Smem& s, const float* f, float (&x)[K0]) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < K0; ++k) x[k] = k >= NFEAT && k < NFEAT + 3 ? 1.f : 0.f;
#pragma unroll
    for (int k = 0; k < NFEAT; ++k) {
        const float v = (f[k] - s.w.lo[k]) * s.w.inv[k];
        ok = ok && (v >= 0.f && v <= 1.f);
        x[k] = v;
    }
    return ok;
}

// CTA set-up: TMEM columns and the mbarrier.
__device__ void cta_setup(Smem& s, uint32_t ncols) {
    if (threadIdx.x < 32) tmem_alloc(&s.tmem, ncols);
    if (threadIdx.x == 0) {
        mbar_init(&s.bar, 1);
        s.fail = 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
}

__device__ void cta_teardown(Smem& s, uint32_t ncols, uint64_t* bar2 = nullptr) {
    fence_before();
    __syncthreads();
    fence_after();
    if (s.fail && threadIdx.x == 0) {
        // a wait expired: give the tensor core one more bounded wait for the
        // products still in flight before their TMEM columns are released
        mbar_wait(&s.bar, 0);
        mbar_wait(&s.bar, 1);
        if (bar2) {
            mbar_wait(bar2, 0);
            mbar_wait(bar2, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(s.tmem, ncols);
}

// Dynamic shared memory rounded up to a 1 KB boundary (the launch adds slack).
template <typename S>
__device__ __forceinline__ S& smem_as(unsigned char* raw) {
    const uintptr_t a = ((uintptr_t)raw + 1023) & ~(uintptr_t)1023;
    return *reinterpret_cast<S*>(a);
}

// D[128 x 64] (TMEM columns dcol..dcol+63) = A[128 x 16 nk] B^T with A and
// B K-major core-matrix tiles of K = 16 nk, issued from thread 0 after the
// CTA's operand stores (and its reads of the columns the product
// overwrites); completion arrives at `bar`.
__device__ void gemm_issue(Smem& s, uint64_t* bar, uint32_t dcol, const unsigned char* A, const unsigned char* B,
                           int nk) {
    fence_async_smem();   // make this thread's shared-memory stores visible to the tensor core
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0) {
        const uint32_t sbo = (uint32_t)nk * 256;   // (K / 8) core matrices of 128 bytes per 8-row group
        for (int kk = 0; kk < nk; ++kk)
            umma(s.tmem + dcol, sdesc(saddr(A) + kk * 256, 128, sbo), sdesc(saddr(B) + kk * 256, 128, sbo),
                 idesc_bf16(TILE, H), kk > 0);
        umma_commit(bar);
    }
}

// Bounded wait for the product committed to `bar` (phase parity `phase`,
// flipped here).  Returns false (and marks the CTA failed) if the wait
// expires; the whole CTA agrees.
__device__ bool gemm_wait(Smem& s, uint64_t* bar, uint32_t& phase, unsigned long long* status) {
    const bool mine = mbar_wait(bar, phase);
    phase ^= 1u;
    const bool failed = __syncthreads_or(!mine) != 0;
    if (failed && threadIdx.x == 0) {
        s.fail = 1;
        atomicAdd(&status[ST_TIMEOUT], 1ull);
        atomicOr(&status[ST_FLAGS], (unsigned long long)CG_FLAG_TIMEOUT);
    }
    fence_after();
    return !failed;
}

__device__ bool run_gemm(Smem& s, uint32_t dcol, const unsigned char* A, const unsigned char* B, int nk,
                         uint32_t& phase, unsigned long long* status) {
    gemm_issue(s, &s.bar, dcol, A, B, nk);
    return gemm_wait(s, &s.bar, phase, status);
}

// The failure path of the bounded waits, without a stalled tensor core: one
// warp waits, with the same bounded wait, on an mbarrier that nothing
// arrives at (phase 0 never completes), and records the expiry in the
// status word exactly as run_gemm does.
__global__ void __launch_bounds__(32) k_wait_selftest(uint32_t polls, unsigned long long* __restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool mine = mbar_wait(&bar, 0, polls);
    const bool failed = __syncthreads_or(!mine) != 0;
    if (failed && threadIdx.x == 0) {
        atomicAdd(&status[ST_TIMEOUT], 1ull);
        atomicOr(&status[ST_FLAGS], (unsigned long long)CG_FLAG_TIMEOUT);
    }
}

// TMEM address of this thread's lane at a column.
__device__ __forceinline__ uint32_t lane_addr(const Smem& s, int col) {
    return s.tmem + ((uint32_t)((threadIdx.x & ~31) & 127) << 16) + (uint32_t)col;
}

// Activation of one value on the CUDA cores (the training kernel's FP32
// path, and the second layer of the ReLU closure) and its derivative.
template <int ACT>
__device__ __forceinline__ float act1(float x) {
    return ACT == ACT_RELU ? fmaxf(x, 0.f) : gelu(x);
}
template <int ACT>
__device__ __forceinline__ float act_grad(float x) {
    return ACT == ACT_RELU ? (x > 0.f ? 1.f : 0.f) : gelu_grad(x);
}

// BF16 act(z) of 16 consecutive columns into row `row` of the second
// product's A tile.  ReLU: the clamp is part of the conversion, one
// instruction per pair.
template <int ACT>
__device__ __forceinline__ void act_store16(unsigned char* A1, int row, int k0, const float (&z)[16]) {
    uint32_t w[8];
    if (ACT == ACT_RELU) {
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = bf16x2_relu(z[2 * i], z[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float a, b;
            gelu2(z[2 * i], z[2 * i + 1], a, b);
            w[i] = bf16x2(a, b);
        }
    }
    *reinterpret_cast<uint4*>(A1 + koff(row, k0, KA)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(A1 + koff(row, k0 + 8, KA)) = make_uint4(w[4], w[5], w[6], w[7]);
}

// First epilogue: act(Z1) of this thread's row (TMEM columns col0..col0+63)
// into the second product's A tile.  The column loops stay rolled: 16
// activations per pass give enough independent work, and the unrolled
// body would not fit the instruction cache beside the rest of the fused
// drag kernel.
template <int ACT>
__device__ __forceinline__ void layer1_epilogue(Smem& s, uint32_t col0) {
#pragma unroll 1
    for (int q = 0; q < H / 16; ++q) {
        float z[16];
        tmem_ld16(lane_addr(s, col0 + 16 * q), z);
        act_store16<ACT>(s.A1, threadIdx.x, 16 * q, z);
    }
}

// Second epilogue: c = act(Z2) w3 + b3 of this thread's row (Z2 in TMEM
// columns col0..col0+63), in FP32.
template <int ACT>
__device__ __forceinline__ float layer2_epilogue(const Smem& s, uint32_t col0) {
    float acc = s.w.b3;
#pragma unroll 1
    for (int q = 0; q < H / 16; ++q) {
        float z[16];
        tmem_ld16(lane_addr(s, col0 + 16 * q), z);
        if (ACT == ACT_RELU) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc = fmaf(fmaxf(z[i], 0.f), s.w.w3[16 * q + i], acc);
        } else {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                float g0, g1;
                gelu2(z[i], z[i + 1], g0, g1);
                acc = fmaf(g0, s.w.w3[16 * q + i], acc);
                acc = fmaf(g1, s.w.w3[16 * q + i + 1], acc);
            }
        }
    }
    return acc;
}

// Forward of the tile: rows' X already in s.X.  Z1 (bias included) goes to
// TMEM columns 0..63 and Z2 to z2col..z2col+63 (0 reuses Z1's columns,
// which are read out before GEMM 2 is issued); returns this thread's c.
template <int ACT>
__device__ bool tile_forward(Smem& s, uint32_t& phase, unsigned long long* status, float& c, uint32_t z2col) {
    if (!run_gemm(s, 0, s.X, s.w.W1t, K0 / 16, phase, status)) return false;
    layer1_epilogue<ACT>(s, 0);
    if (!run_gemm(s, z2col, s.A1, s.w.W2t, KA / 16, phase, status)) return false;
    c = layer2_epilogue<ACT>(s, z2col);
    return true;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// c for every feature row (rows outside the training box still get c; the
// in-range flag tells the caller).
template <int ACT>
__global__ void __launch_bounds__(TILE, 4)
k_mlp_forward(const WeightImage* __restrict__ img, const float* __restrict__ feat, long long n,
              float* __restrict__ c_out, int32_t* __restrict__ in_range, unsigned long long* __restrict__ status) {
    pdl_wait();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Smem& s = smem_as<Smem>(smem_raw);
    load_weights(s, img);
    cta_setup(s, kInferCols);
    uint32_t phase = 0;
    const long long ntiles = (n + TILE - 1) / TILE;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long r = t * TILE + threadIdx.x;
        float f[FEAT_STRIDE] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (r < n) {
            const float4 a = reinterpret_cast<const float4*>(feat)[2 * r];
            const float4 b = reinterpret_cast<const float4*>(feat)[2 * r + 1];
            f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
        }
        float x[K0];
        const bool ok = scale_row(s, f, x);
        st_row8(s.X, threadIdx.x, 0, K0, x);
        st_row8(s.X, threadIdx.x, 8, K0, x + 8);
        float c = 0.f;
        if (!tile_forward<ACT>(s, phase, status, c, 0)) break;
        if (r < n) {
            c_out[r] = c;
            if (in_range) in_range[r] = ok ? 1 : 0;
        }
    }
    cta_teardown(s, kInferCols);
}

// Loss and gradient partials of a batch: each CTA accumulates its tiles'
// contributions in a fixed order and writes one partial per parameter.
// Layout of part: [gridDim.x][NPARAM + 1] (the last entry: sum of residual^2).
template <int ACT>
__global__ void __launch_bounds__(TILE, 1)
k_mlp_grad(const float* __restrict__ P, const WeightImage* __restrict__ img, const float* __restrict__ feat,
           const float* __restrict__ target, long long n, float* __restrict__ part,
           unsigned long long* __restrict__ status) {
    pdl_wait();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    SmemTrain& st = smem_as<SmemTrain>(smem_raw);
    Smem& s = st.s;
    load_weights(s, img);
    load_w2b(st, P);
    cta_setup(s, kTrainCols);
    uint32_t phase = 0;
    const int tid = threadIdx.x;
    const float inv_n = 1.0f / (float)n;
    // this thread's gradient accumulators: W2 entries tid*32 .. +32 (flattened
    // (in, out)), W1 entries tid*8 .. +8, bias / w3 entries for tid < 64
    float gW2[32], gW1[8];
#pragma unroll
    for (int i = 0; i < 32; ++i) gW2[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) gW1[i] = 0.f;
    float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, loss = 0.f;
    const long long ntiles = (n + TILE - 1) / TILE;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long r = t * TILE + tid;
        float f[FEAT_STRIDE] = {0, 0, 0, 0, 0, 0, 0, 0};
        float tg = 0.f;
        if (r < n) {
            const float4 a = reinterpret_cast<const float4*>(feat)[2 * r];
            const float4 b = reinterpret_cast<const float4*>(feat)[2 * r + 1];
            f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
            tg = target[r];
        }
        float x[K0];
        scale_row(s, f, x);
        st_row8(s.X, tid, 0, K0, x);
        st_row8(s.X, tid, 8, K0, x + 8);
        float c = 0.f;
        if (!tile_forward<ACT>(s, phase, status, c, 64)) break;
        const float res = (r < n) ? (c - tg) : 0.f;
        const float dc = 2.0f * res * inv_n;
        st.dc[tid] = dc;
        st.r2[tid] = res * res;
        // dZ2 = dc w3 * act'(Z2); A2 dc for the w3 gradient
#pragma unroll
        for (int q = 0; q < H / 16; ++q) {
            float z[16], d[16];
            tmem_ld16(lane_addr(s, 64 + 16 * q), z);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int j = 16 * q + i;
                d[i] = dc * s.w.w3[j] * act_grad<ACT>(z[i]);
                st.dZ2[tid][j] = d[i];
                st.A2dc[tid][j] = act1<ACT>(z[i]) * dc;
            }
            st_row8(st.dZ2b, tid, 16 * q, H, d);
            st_row8(st.dZ2b, tid, 16 * q + 8, H, d + 8);
        }
        // dA1 = dZ2 W2^T on the tensor cores
        if (!run_gemm(s, 128, st.dZ2b, st.W2b, H / 16, phase, status)) break;
#pragma unroll
        for (int q = 0; q < H / 16; ++q) {
            float da[16], z1[16];
            tmem_ld16(lane_addr(s, 128 + 16 * q), da);
            tmem_ld16(lane_addr(s, 16 * q), z1);
#pragma unroll
            for (int i = 0; i < 16; ++i) st.dZ1[tid][16 * q + i] = da[i] * act_grad<ACT>(z1[i]);
        }
        __syncthreads();
        // weight gradients, rows summed in increasing order
#pragma unroll 1
        for (int row = 0; row < TILE; ++row) {
            // W2 (in, out): entries tid*32 + e -> in = (tid*32+e) / 64, out = (tid*32+e) % 64
            const int in = (tid * 32) / H, out0 = (tid * 32) % H;
            const float a1 = bf16_val(*reinterpret_cast<const uint16_t*>(s.A1 + koff(row, in, KA)));
#pragma unroll
            for (int e = 0; e < 32; ++e) gW2[e] = fmaf(a1, st.dZ2[row][out0 + e], gW2[e]);
            // W1 (k, j): entries tid*8 + e -> k = (tid*8+e) / 64, j = (tid*8+e) % 64; the
            // inputs past NFEAT are zero in the network (the tile's ones there meet b1)
            const int k = (tid * 8) / H, j0 = (tid * 8) % H;
            const float xk =
                k < NFEAT ? bf16_val(*reinterpret_cast<const uint16_t*>(s.X + koff(row, k, K0))) : 0.f;
#pragma unroll
            for (int e = 0; e < 8; ++e) gW1[e] = fmaf(xk, st.dZ1[row][j0 + e], gW1[e]);
            if (tid < H) {
                gb1 += st.dZ1[row][tid];
                gb2 += st.dZ2[row][tid];
                gw3 += st.A2dc[row][tid];
            } else if (tid == H) {
                gb3 += st.dc[row];
                loss += st.r2[row];
            }
        }
        __syncthreads();
    }
    float* out = part + (long long)blockIdx.x * (NPARAM + 1);
#pragma unroll
    for (int e = 0; e < 32; ++e) out[OFF_W2 + tid * 32 + e] = gW2[e];
#pragma unroll
    for (int e = 0; e < 8; ++e) out[OFF_W1 + tid * 8 + e] = gW1[e];
    if (tid < H) {
        out[OFF_B1 + tid] = gb1;
        out[OFF_B2 + tid] = gb2;
        out[OFF_W3 + tid] = gw3;
    } else if (tid == H) {
        out[OFF_B3] = gb3;
        out[NPARAM] = loss;
    }
    cta_teardown(s, kTrainCols);
}

// Sum the CTA partials (fixed order), optionally apply one Adam step.
__global__ void __launch_bounds__(256)
k_mlp_reduce_adam(const float* __restrict__ part, int nparts, float* __restrict__ grads, float* __restrict__ P,
                  float* __restrict__ m, float* __restrict__ v, int t, float lr, int do_update,
                  float* __restrict__ loss_out, long long n) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > NPARAM) return;
    float g = 0.f;
    for (int b = 0; b < nparts; ++b) g += part[(long long)b * (NPARAM + 1) + i];
    if (i == NPARAM) {
        if (loss_out) loss_out[0] = g / (float)n;
        return;
    }
    grads[i] = g;
    if (do_update) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / (1.f - powf(b1, (float)t));
        const float vh = vi / (1.f - powf(b2, (float)t));
        P[i] -= lr * mh / (sqrtf(vh) + eps);
    }
}

// ---------------------------------------------------------------------------
// Closure inputs and training targets at every particle (any precision):
// features from the stale bulk record (porosity of this step, velocity and
// variance of the last refresh), target c* = (F_fresh . F_stale) / |F_stale|^2.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void closure_features(const Probe<T>& st, const V4<T>& x, const V4<T>& v,
                                                 const GridDev& g, const Phys<T>& P, float (&f)[FEAT_STRIDE],
                                                 T& epsc, T& phic, T (&s)[3], T& smag) {
    const T eps = st.eps;
    epsc = eps;
    phic = T(1) - eps;
    if (eps < P.eps_min) {
        epsc = P.eps_min;
        phic = T(1) - P.eps_min;
    }
    s[0] = st.ux - v.x;
    s[1] = st.uy - v.y;
    s[2] = st.uz - v.z;
    smag = M<T>::sqrt_(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    const T Re = P.rho_mu * epsc * x.w * smag;
    f[0] = (float)epsc;
    f[1] = (float)(sizeof(T) == 4 ? log10f((float)(T(1) + Re)) : log10((double)(T(1) + Re)));
    f[2] = (float)smag;
    f[3] = (float)st.geps[0];
    f[4] = (float)st.geps[1];
    f[5] = (float)st.geps[2];
    f[6] = (float)st.sc;
    f[7] = 0.f;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_mlp_features(const T* __restrict__ pos, const T* __restrict__ vel, long long n, GridDev g, Phys<T> P,
               const T* __restrict__ bulk_stale, const T* __restrict__ var_stale, const T* __restrict__ bulk_fresh,
               float* __restrict__ feat, float* __restrict__ target) {
    pdl_wait();
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const V4<T> x = ld4(pos, p), v = ld4(vel, p);
        const Probe<T> st = probe(bulk_stale, var_stale, x.x, x.y, x.z, g);
        const V4<T> fr = gather(bulk_fresh, x.x, x.y, x.z, g);
        float f[FEAT_STRIDE];
        T epsc, phic, s[3], smag;
        closure_features(st, x, v, g, P, f, epsc, phic, s, smag);
        const T bs = drag_beta(g.law, epsc, phic, x.w, smag, P);
        const T sf[3] = {fr.y - v.x, fr.z - v.y, fr.w - v.z};
        const T sfm = M<T>::sqrt_(sf[0] * sf[0] + sf[1] * sf[1] + sf[2] * sf[2]);
        const T bf = drag_beta(g.law, epsc, phic, x.w, sfm, P);
        T dot = 0, nn = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T Fs = bs * s[a], Ff = bf * sf[a];
            dot += Ff * Fs;
            nn += Fs * Fs;
        }
        reinterpret_cast<float4*>(feat)[2 * p] = make_float4(f[0], f[1], f[2], f[3]);
        reinterpret_cast<float4*>(feat)[2 * p + 1] = make_float4(f[4], f[5], f[6], 0.f);
        target[p] = nn > T(0) ? (float)(dot / nn) : 1.0f;
    }
}

// Fresh fluid velocity at a point averaged on demand from the fine grid
// (the fallback of the learned drag): mean of the r^3 fine cells of each
// bulk cell the stencil touches, then the same interpolation as the gather.
__device__ V4<float> fresh_velocity(const float* __restrict__ u_fine, float x, float y, float z, const GridDev& g) {
    int i0[3] = {0, 0, 0};
    float t[3] = {0.f, 0.f, 0.f};
    const bool cell = g.interp == CG_INTERP_CELL;
    if (cell) {
        const int c = cell_of_f(x, y, z, g);
        i0[0] = c % g.nb[0];
        i0[1] = (c / g.nb[0]) % g.nb[1];
        i0[2] = c / (g.nb[0] * g.nb[1]);
    } else {
        axis_weight(x, g, 0, i0[0], t[0]);
        axis_weight(y, g, 1, i0[1], t[1]);
        axis_weight(z, g, 2, i0[2], t[2]);
    }
    const int r = g.r;
    const long long nx = g.nf[0], nxy = (long long)g.nf[0] * g.nf[1];
    const float inv = 1.0f / (float)(r * r * r);
    // per-axis pair of bulk values, interpolated x, then y, then z as the gather does
    float corner[8][3];
    for (int q = 0; q < (cell ? 1 : 8); ++q) {
        const int I = i0[0] + (q & 1), J = i0[1] + ((q >> 1) & 1), K = i0[2] + (q >> 2);
        float sum[3] = {0.f, 0.f, 0.f};
        for (int dk = 0; dk < r; ++dk)
            for (int dj = 0; dj < r; ++dj) {
                const long long row = nx * (J * r + dj) + nxy * (K * r + dk) + (long long)I * r;
                for (int di = 0; di < r; ++di)
                    for (int c = 0; c < 3; ++c) sum[c] += __ldg(u_fine + c * g.nfine + row + di);
            }
        for (int c = 0; c < 3; ++c) corner[q][c] = sum[c] * inv;
    }
    if (cell) return {0.f, corner[0][0], corner[0][1], corner[0][2]};
    float u[3];
    for (int c = 0; c < 3; ++c) {
        const float a00 = lerp_(corner[0][c], corner[1][c], t[0]), a10 = lerp_(corner[2][c], corner[3][c], t[0]);
        const float a01 = lerp_(corner[4][c], corner[5][c], t[0]), a11 = lerp_(corner[6][c], corner[7][c], t[0]);
        u[c] = lerp_(lerp_(a00, a10, t[1]), lerp_(a01, a11, t[1]), t[2]);
    }
    return {0.f, u[0], u[1], u[2]};
}

// Shared memory of the learned drag: the forward part, a second mbarrier
// (completions of the second product) and, for the tile between its two
// halves, each row's state in a thread-private stash (two tiles deep).
struct SmemLearned {
    Smem s;
    uint64_t bar2;
    float4 x[2][TILE], v[2][TILE];   // position and velocity as read
    float4 F[2][TILE];               // stale drag (fallback rows: the drag itself); w = sorted slot
    int state[2][TILE];              // 0 no row, 1 learned, 2 fallback
};
constexpr uint32_t kLearnCols = 128;    // Z of two tiles in flight: columns 0..63 and 64..127

// Learned drag: per tile of 128 particles (caller order) each thread forms
// its particle's closure inputs and the drag F_stale from the stale bulk
// record (porosity of this step, fluid velocity and variance of the last
// refresh, `age` steps ago); the tile goes through the network on the
// tensor cores, whose output r is the correction per step; in range
// F = (1 + age r) F_stale, otherwise F is the plain drag with the fluid
// velocity averaged afresh from the fine grid.  The force is also written
// to its sorted slot for the fused reaction deposit when Fs is given, and
// with dt > 0 the particle is advanced as the plain drag kernel does.
//
// Software pipeline over a CTA's tiles t (two TMEM buffers, b = tile
// parity): (A) rows of t: inputs (loaded one tile ahead), features, stale
// drag; issue the first product of t; load the inputs of the next tile;
// (B) wait for the second product of t - 1, its output c and the stores of
// t - 1; (C) wait for the first product of t, the activations, issue the
// second product of t.  The first product runs under (B), the second
// under the next (A).
template <int ACT>
__global__ void __launch_bounds__(TILE, 4)
k_drag_learned(float* pos, float* vel, long long n, GridDev g, Phys<float> P, const float* __restrict__ bulk_stale,
               const float* __restrict__ var_stale, const float* __restrict__ u_fine,
               const WeightImage* __restrict__ img, float* __restrict__ F, float* __restrict__ Fs,
               const int32_t* __restrict__ inv_perm, float dt, float age, unsigned long long* __restrict__ status) {
    pdl_wait();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    SmemLearned& L = smem_as<SmemLearned>(smem_raw);
    Smem& s = L.s;
    const int tid = threadIdx.x;
    load_weights(s, img);
    if (tid == 0) mbar_init(&L.bar2, 1);
    cta_setup(s, kLearnCols);
    uint32_t ph1 = 0, ph2 = 0;
    unsigned fallbacks = 0, clamped = 0;
    const long long ntiles = (n + TILE - 1) / TILE;
    // this thread's row of the coming tile, loaded a tile ahead
    float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), va = xa;
    int slot = 0;
    auto fetch = [&](long long t) {
        const long long p = t * TILE + tid;
        if (t < ntiles && p < n) {
            xa = reinterpret_cast<const float4*>(pos)[p];
            va = reinterpret_cast<const float4*>(vel)[p];
            slot = Fs ? __ldg(inv_perm + p) : 0;
        }
    };
    fetch(blockIdx.x);
    long long prev = -1;
    int b = 0;
    for (long long t = blockIdx.x;; t += gridDim.x) {
        const bool have = t < ntiles;
        if (have) {
            // (A) rows of tile t
            const long long p = t * TILE + tid;
            float f[FEAT_STRIDE] = {0, 0, 0, 0, 0, 0, 0, 0};
            float Fo[3] = {0.f, 0.f, 0.f};
            float epsc = 1.f, phic = 0.f;
            if (p < n) {
                const Probe<float> st = probe(bulk_stale, var_stale, xa.x, xa.y, xa.z, g);
                const V4<float> x = {xa.x, xa.y, xa.z, xa.w}, v = {va.x, va.y, va.z, va.w};
                float sv[3], smag;
                closure_features(st, x, v, g, P, f, epsc, phic, sv, smag);
                clamped += st.eps < P.eps_min;
                const float be = drag_beta(g.law, epsc, phic, xa.w, smag, P);
                Fo[0] = be * sv[0];
                Fo[1] = be * sv[1];
                Fo[2] = be * sv[2];
            }
            float xin[K0];
            const bool ok = scale_row(s, f, xin);
            st_row8(s.X, tid, 0, K0, xin);
            st_row8(s.X, tid, 8, K0, xin + 8);
            if (p < n && !ok) {
                // out of the training box: the plain drag with the fluid velocity averaged afresh
                ++fallbacks;
                const V4<float> uf = fresh_velocity(u_fine, xa.x, xa.y, xa.z, g);
                const float sf[3] = {uf.y - va.x, uf.z - va.y, uf.w - va.z};
                const float sm = sqrtf(sf[0] * sf[0] + sf[1] * sf[1] + sf[2] * sf[2]);
                const float be = drag_beta(g.law, epsc, phic, xa.w, sm, P);
                Fo[0] = be * sf[0];
                Fo[1] = be * sf[1];
                Fo[2] = be * sf[2];
            }
            L.x[b][tid] = xa;
            L.v[b][tid] = va;
            L.F[b][tid] = make_float4(Fo[0], Fo[1], Fo[2], __int_as_float(slot));
            L.state[b][tid] = p < n ? (ok ? 1 : 2) : 0;
            gemm_issue(s, &s.bar, (uint32_t)b * 64, s.X, s.w.W1t, K0 / 16);
            fetch(t + gridDim.x);
        }
        if (prev >= 0) {
            // (B) tile prev: its second product, c, the outputs
            if (!gemm_wait(s, &L.bar2, ph2, status)) break;
            const int pb = b ^ 1;
            const float c = layer2_epilogue<ACT>(s, (uint32_t)pb * 64);
            const int state = L.state[pb][tid];
            if (state) {
                const long long p = prev * TILE + tid;
                const float4 Fv = L.F[pb][tid];
                const float cc = state == 1 ? fmaf(age, c, 1.0f) : 1.0f;   // correction after `age` steps
                const float Fo[3] = {cc * Fv.x, cc * Fv.y, cc * Fv.z};
                F[p] = Fo[0];
                F[n + p] = Fo[1];
                F[2 * n + p] = Fo[2];
                if (Fs) st4(Fs, __float_as_int(Fv.w), Fo[0], Fo[1], Fo[2], 0.f);
                if (dt > 0.f) {
                    const float4 x = L.x[pb][tid], v = L.v[pb][tid];
                    const float m = P.rho_p * M<float>::pi6() * x.w * x.w * x.w;
                    float xn[3] = {x.x, x.y, x.z};
                    float un[3] = {v.x + dt * (Fo[0] / m + P.g[0]), v.y + dt * (Fo[1] / m + P.g[1]),
                                   v.z + dt * (Fo[2] / m + P.g[2])};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        float xq = xn[a] + dt * un[a];
                        const float lo = g.x0f[a], hi = g.xhif[a];
                        if (xq < lo) { xq = 2.f * lo - xq; un[a] = -un[a]; }
                        else if (xq > hi) { xq = 2.f * hi - xq; un[a] = -un[a]; }
                        xn[a] = xq;
                    }
                    st4(pos, p, xn[0], xn[1], xn[2], x.w);
                    st4(vel, p, un[0], un[1], un[2], v.w);
                }
            }
        }
        if (!have) break;
        // (C) tile t: first product, activations, second product
        if (!gemm_wait(s, &s.bar, ph1, status)) break;
        layer1_epilogue<ACT>(s, (uint32_t)b * 64);
        gemm_issue(s, &L.bar2, (uint32_t)b * 64, s.A1, s.w.W2t, KA / 16);
        prev = t;
        b ^= 1;
    }
    if (fallbacks) atomicAdd(&status[ST_FALLBACK], (unsigned long long)fallbacks);
    if (clamped) {
        atomicAdd(&status[ST_CLAMPED], (unsigned long long)clamped);
        atomicOr(&status[ST_FLAGS], (unsigned long long)CG_FLAG_EPS_CLAMPED);
    }
    cta_teardown(s, kLearnCols, &L.bar2);
}

}  // namespace mlp
}  // namespace cg

// ---------------------------------------------------------------------------
// Handle and C ABI
// ---------------------------------------------------------------------------
struct cg_mlp {
    cudaStream_t stream = nullptr;
    int num_sms = 148;
    float* P = nullptr;        // FP32 master parameters
    float* m = nullptr;        // Adam first moments
    float* v = nullptr;        // Adam second moments
    float* grads = nullptr;    // last reduced gradient
    float* scale = nullptr;    // lo[8], 1/(hi - lo)[8]
    cg::mlp::WeightImage* img = nullptr;   // the forward operands, rebuilt whenever P changes
    float* part = nullptr;     // CTA partials
    unsigned long long* status = nullptr;
    float lo[8] = {0}, hi[8] = {0};
    int t = 0;
    const void* var_bulk = nullptr;   // bound inputs of the fused learned drag
    const void* u_fine = nullptr;
    int32_t age = 1;
    int32_t act = CG_MLP_GELU;        // activation of both hidden layers
};

namespace {
using namespace cg::mlp;

// Forward-only CTAs hold 64 TMEM columns each and at least 28 KB of shared
// memory, so at most eight share an SM and their columns always fit in the
// SM's 512 (a training CTA, 256 columns and over 150 KB, leaves room for at
// most two of them beside it).
size_t smem_forward() { return std::max<size_t>(sizeof(Smem) + 1024, 28 * 1024); }
// A learned-drag CTA holds 128 TMEM columns: its shared memory (over 46 KB)
// keeps it to four per SM, whose columns fill the SM's 512 at most.
size_t smem_learned() { return std::max<size_t>(sizeof(SmemLearned) + 1024, 47 * 1024); }
size_t smem_train() { return sizeof(SmemTrain) + 1024; }
cg::PerDeviceOnce g_mlp_attr_once;

template <int ACT>
cudaError_t mlp_attrs_of() {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward<ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_forward());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_grad<ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_train());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_drag_learned<ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_learned());
    return e;
}

cg_status mlp_attrs() {
    return cg::once_per_device(g_mlp_attr_once, [] {
        CG_CUDA(mlp_attrs_of<ACT_GELU>());
        CG_CUDA(mlp_attrs_of<ACT_RELU>());
        return CG_OK;
    });
}

// Rebuild the weight image from P on the closure's stream (after every
// change of P, in the same stream order).
cg_status rebuild_image(cg_mlp* m) {
    k_mlp_image<<<1, 256, 0, m->stream>>>(m->P, m->scale, m->img);
    CG_CUDA(cudaGetLastError());
    return CG_OK;
}

void host_scale(const float* lo, const float* hi, float out[16]) {
    for (int k = 0; k < 8; ++k) {
        out[k] = lo[k];
        const float r = hi[k] - lo[k];
        out[8 + k] = r > 0.f ? 1.0f / r : 0.f;
    }
}

}  // namespace

namespace cg {

cg_status mlp_bound_inputs(const cg_mlp* m, const void** var_stale, const void** u_fine, int32_t* age) {
    if (!m->var_bulk || !m->u_fine) return CG_ERR_INVALID_ARG;
    *var_stale = m->var_bulk;
    *u_fine = m->u_fine;
    *age = m->age;
    return CG_OK;
}

cg_status launch_drag_learned(cg_grids* g, const cg_mlp* m, long long n, void* pos_d, void* vel,
                              const void* var_stale, const void* u_fine, int32_t age, void* force, void* S_bulk,
                              double dt) {
    if (g->fp64 || !var_stale || !u_fine || age < 1) return CG_ERR_INVALID_ARG;
    if (n > 0 && ((uintptr_t)u_fine & 15u)) return CG_ERR_INVALID_ARG;
    CG_TRY(mlp_attrs());
    g->part_blocks[PS_DRAG] = -1;   // the drag diagnostics are not formed on this path
    void* Fs = S_bulk ? g->Fs : nullptr;
    if (n > 0) {
        const long long ntiles = (n + TILE - 1) / TILE;
        const unsigned grid = (unsigned)std::min(ntiles, (long long)4 * g->num_sms);
        auto kern = m->act == CG_MLP_RELU ? k_drag_learned<ACT_RELU> : k_drag_learned<ACT_GELU>;
        CG_LAUNCH(g, "drag_learned", kern, grid, TILE, smem_learned(), (float*)pos_d, (float*)vel, n, g->gd,
                  cg::phys_of<float>(g->gd), (const float*)g->bulk4, (const float*)var_stale, (const float*)u_fine,
                  (const WeightImage*)m->img, (float*)force, (float*)Fs, g->inv_perm, (float)dt, (float)age,
                  g->status);
    }
    if (S_bulk) CG_TRY(launch_deposit_sorted_force(g, n, S_bulk));
    return CG_OK;
}

}  // namespace cg

namespace cg {
cg_status mlp_feature_box(const cg_mlp* m, float* lo, float* hi) {
    if (!m) return CG_ERR_INVALID_ARG;
    for (int k = 0; k < NFEAT; ++k) {
        lo[k] = m->lo[k];
        hi[k] = m->hi[k];
    }
    return CG_OK;
}
}  // namespace cg

extern "C" {

cg_status cg_mlp_features(cg_grids* g, int64_t n, const void* pos_d, const void* vel, const double* eps_bulk,
                          const void* u_stale, const void* var_stale, const void* u_fresh, float* feat_out,
                          float* target_out) {
    if (!g) return CG_ERR_INVALID_ARG;
    if (n < 0 || n > INT32_MAX) return CG_ERR_INVALID_ARG;
    if (!eps_bulk || !u_stale || !var_stale || !u_fresh) return CG_ERR_INVALID_ARG;
    if (n > 0 && (!pos_d || !vel || !feat_out || !target_out)) return CG_ERR_INVALID_ARG;
    if (n > 0 && (((uintptr_t)pos_d | (uintptr_t)vel | (uintptr_t)feat_out) & 15u)) return CG_ERR_INVALID_ARG;
    // pack (phi, u_fresh) into the fresh record, then (phi, u_stale) into the drag's record
    void* const keep = g->bulk4;
    CG_TRY(grow_buf(g->fresh4, 4 * g->tsize * (size_t)g->gd.nbulk));
    g->bulk4 = g->fresh4.p;
    const cg_status s1 = cg::launch_pack(g, eps_bulk, u_fresh, false);
    g->bulk4 = keep;
    CG_TRY(s1);
    CG_TRY(cg::launch_pack(g, eps_bulk, u_stale, false));
    if (n == 0) return CG_OK;
    const unsigned grid = (unsigned)std::min((n + 255) / 256, (int64_t)g->num_sms * 8);
    if (g->fp64)
        CG_LAUNCH(g, "mlp_features", k_mlp_features<double>, grid, 256, 0, (const double*)pos_d, (const double*)vel,
                  (long long)n, g->gd, cg::phys_of<double>(g->gd), (const double*)g->bulk4, (const double*)var_stale,
                  (const double*)g->fresh4.p, feat_out, target_out);
    else
        CG_LAUNCH(g, "mlp_features", k_mlp_features<float>, grid, 256, 0, (const float*)pos_d, (const float*)vel,
                  (long long)n, g->gd, cg::phys_of<float>(g->gd), (const float*)g->bulk4, (const float*)var_stale,
                  (const float*)g->fresh4.p, feat_out, target_out);
    return CG_OK;
}

cg_status cg_mlp_bind(cg_mlp* m, const void* var_stale, const void* u_fine, int32_t age) {
    if (!m) return CG_ERR_INVALID_ARG;
    if ((var_stale == nullptr) != (u_fine == nullptr) || ((uintptr_t)u_fine & 15u)) return CG_ERR_INVALID_ARG;
    if (var_stale && age < 1) return CG_ERR_INVALID_ARG;
    m->var_bulk = var_stale;
    m->u_fine = u_fine;
    m->age = var_stale ? age : 1;
    return CG_OK;
}

cg_status cg_mlp_create(const float* params, const float* feat_lo, const float* feat_hi, void* cuda_stream,
                        cg_mlp** out) {
    if (!out) return CG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || !feat_lo || !feat_hi) return CG_ERR_INVALID_ARG;
    for (int k = 0; k < NFEAT; ++k)
        if (!(feat_hi[k] > feat_lo[k]) || !isfinite(feat_lo[k]) || !isfinite(feat_hi[k])) return CG_ERR_INVALID_ARG;
    cg_mlp* m = new (std::nothrow) cg_mlp();
    if (!m) return CG_ERR_OOM;
    m->stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
    for (int k = 0; k < 8; ++k) {
        m->lo[k] = k < NFEAT ? feat_lo[k] : 0.f;
        m->hi[k] = k < NFEAT ? feat_hi[k] : 1.f;
    }
    float sc[16];
    host_scale(m->lo, m->hi, sc);
    const size_t pb = sizeof(float) * NPARAM;
    const size_t partb = sizeof(float) * (size_t)(NPARAM + 1) * (size_t)(2 * m->num_sms);
    bool ok = cudaMalloc(&m->P, pb) == cudaSuccess && cudaMalloc(&m->m, pb) == cudaSuccess &&
              cudaMalloc(&m->v, pb) == cudaSuccess && cudaMalloc(&m->grads, pb) == cudaSuccess &&
              cudaMalloc(&m->scale, sizeof sc) == cudaSuccess && cudaMalloc(&m->part, partb) == cudaSuccess &&
              cudaMalloc(&m->img, sizeof(WeightImage)) == cudaSuccess &&
              cudaMalloc(&m->status, sizeof(unsigned long long) * cg::kNumSlots) == cudaSuccess;
    ok = ok && cudaMemcpy(m->P, params, pb, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(m->m, 0, pb) == cudaSuccess && cudaMemset(m->v, 0, pb) == cudaSuccess &&
         cudaMemcpy(m->scale, sc, sizeof sc, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(m->status, 0, sizeof(unsigned long long) * cg::kNumSlots) == cudaSuccess;
    ok = ok && mlp_attrs() == CG_OK && rebuild_image(m) == CG_OK && cudaStreamSynchronize(m->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(m->P); cudaFree(m->m); cudaFree(m->v); cudaFree(m->grads); cudaFree(m->scale);
        cudaFree(m->part); cudaFree(m->status); cudaFree(m->img);
        delete m;
        return CG_ERR_OOM;
    }
    *out = m;
    return CG_OK;
}

cg_status cg_mlp_destroy(cg_mlp* m) {
    if (!m) return CG_OK;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->P); cudaFree(m->m); cudaFree(m->v); cudaFree(m->grads); cudaFree(m->scale);
    cudaFree(m->part); cudaFree(m->status); cudaFree(m->img);
    cudaGetLastError();
    delete m;
    return CG_OK;
}


cg_status cg_mlp_get_params(cg_mlp* m, float* params, float* grads) {
    if (!m) return CG_ERR_INVALID_ARG;
    CG_CUDA(cudaStreamSynchronize(m->stream));
    if (params) CG_CUDA(cudaMemcpy(params, m->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    if (grads) CG_CUDA(cudaMemcpy(grads, m->grads, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    return CG_OK;
}

cg_status cg_mlp_set_activation(cg_mlp* m, int32_t activation) {
    if (!m || (activation != CG_MLP_GELU && activation != CG_MLP_RELU)) return CG_ERR_INVALID_ARG;
    m->act = activation;
    return CG_OK;
}

cg_status cg_mlp_get_activation(const cg_mlp* m, int32_t* activation) {
    if (!m || !activation) return CG_ERR_INVALID_ARG;
    *activation = m->act;
    return CG_OK;
}

cg_status cg_mlp_set_params(cg_mlp* m, const float* params) {
    if (!m || !params) return CG_ERR_INVALID_ARG;
    CG_CUDA(cudaMemcpyAsync(m->P, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, m->stream));
    CG_TRY(rebuild_image(m));
    CG_CUDA(cudaStreamSynchronize(m->stream));
    return CG_OK;
}

cg_status cg_mlp_forward(cg_mlp* m, int64_t n, const float* features, float* c_out, int32_t* in_range_out) {
    if (!m || n < 0 || (n > 0 && (!features || !c_out || ((uintptr_t)features & 15u)))) return CG_ERR_INVALID_ARG;
    if (n == 0) return CG_OK;
    CG_TRY(mlp_attrs());
    const long long ntiles = (n + TILE - 1) / TILE;
    const unsigned grid = (unsigned)std::min(ntiles, (long long)4 * m->num_sms);
    auto kern = m->act == CG_MLP_RELU ? k_mlp_forward<ACT_RELU> : k_mlp_forward<ACT_GELU>;
    kern<<<grid, TILE, smem_forward(), m->stream>>>(m->img, features, n, c_out, in_range_out, m->status);
    CG_CUDA(cudaGetLastError());
    return CG_OK;
}

static cg_status grad_impl(cg_mlp* m, int64_t n, const float* features, const float* targets, float lr,
                           int do_update, float* loss_out) {
    if (!m || n <= 0 || !features || !targets || ((uintptr_t)features & 15u)) return CG_ERR_INVALID_ARG;
    CG_TRY(mlp_attrs());
    const long long ntiles = (n + TILE - 1) / TILE;
    const int grid = (int)std::min(ntiles, (long long)m->num_sms);
    auto kern = m->act == CG_MLP_RELU ? k_mlp_grad<ACT_RELU> : k_mlp_grad<ACT_GELU>;
    kern<<<grid, TILE, smem_train(), m->stream>>>(m->P, m->img, features, targets, n, m->part, m->status);
    CG_CUDA(cudaGetLastError());
    if (do_update) m->t += 1;
    k_mlp_reduce_adam<<<(NPARAM + 1 + 255) / 256, 256, 0, m->stream>>>(m->part, grid, m->grads, m->P, m->m, m->v,
                                                                        m->t, lr, do_update, loss_out, n);
    CG_CUDA(cudaGetLastError());
    if (do_update) CG_TRY(rebuild_image(m));
    return CG_OK;
}

cg_status cg_mlp_grads(cg_mlp* m, int64_t n, const float* features, const float* targets, float* loss_out) {
    return grad_impl(m, n, features, targets, 0.f, 0, loss_out);
}

cg_status cg_mlp_train_step(cg_mlp* m, int64_t n, const float* features, const float* targets, float lr,
                            float* loss_out) {
    if (!(lr > 0.f) || !isfinite(lr)) return CG_ERR_INVALID_ARG;
    return grad_impl(m, n, features, targets, lr, 1, loss_out);
}

cg_status cg_mlp_wait_selftest(cg_mlp* m, uint32_t polls) {
    if (!m || polls == 0 || polls > kSpinLimit) return CG_ERR_INVALID_ARG;
    k_wait_selftest<<<1, 32, 0, m->stream>>>(polls, m->status);
    CG_CUDA(cudaGetLastError());
    return CG_OK;
}

cg_status cg_mlp_sync_status(cg_mlp* m, uint32_t* flags) {
    if (!m) return CG_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return CG_ERR_CUDA;
    }
    unsigned long long h[cg::kNumSlots];
    CG_CUDA(cudaMemcpy(h, m->status, sizeof h, cudaMemcpyDeviceToHost));
    CG_CUDA(cudaMemset(m->status, 0, sizeof h));
    if (flags) *flags = (uint32_t)h[cg::ST_FLAGS];
    return (h[cg::ST_FLAGS] & CG_FLAG_TIMEOUT) ? CG_ERR_TIMEOUT : CG_OK;
}

}  // extern "C"
