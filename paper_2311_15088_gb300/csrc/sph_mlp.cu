// sph_mlp.cu -- the boid-force surrogate: a 272 -> 256 -> 256 -> 256 -> 16
// MLP (exact-erf GELU) whose inference and training GEMMs run on the
// tensor cores (tcgen05.mma kind::f16: BF16 operands staged by TMA, FP32
// accumulators in tensor memory), with Adam on FP32 master weights.
//
// The surrogate is not in the paper; it predicts the fluid force the SPH
// coupling of section "Boid Motion and Agent Fluid Interaction" puts on a
// boid (F_b in v_b += sph_factor dt F_b) from the flow around the boid.
//
// Layout: a layer's weight W is [out][in] (K-major for the B operand of the
// forward GEMM) with a transposed BF16 copy W^T [in][out] for the backward
// GEMM; activations are [batch][features] with transposed copies
// [features][batch] for the weight-gradient GEMMs (which contract over the
// batch).  Every GEMM is C[M][N] = A[M][K] . B[N][K]^T with both operands
// K-major.
#include <cudaTypedefs.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>

#include "sph_umma.cuh"

namespace sphk {

constexpr int BM = 128;  // rows per tile (UMMA M)
constexpr int BK = 64;   // K elements per pipeline stage (one 128-byte row)
constexpr int UK = 16;   // K per tcgen05.mma of kind::f16

enum { EPI_BIAS_GELU = 0, EPI_BIAS = 1, EPI_GELU_GRAD = 2, EPI_F32 = 3 };

struct GemmEpi {
    int M, N;                 // valid rows / columns of C
    int kb_total;             // K blocks of BK
    int kb_per_split;         // K blocks per blockIdx.z
    const float* bias;        // [N]
    __nv_bfloat16* out_bf16;  // [M][ld_bf16]
    int ld_bf16;
    __nv_bfloat16* out_t;     // [N][ld_t] (transposed copy)
    int ld_t;
    float* out_f32;           // [M][ld_f32] (+ blockIdx.z * split_stride for EPI_F32)
    int ld_f32;
    long long split_stride;
    const float* zin;         // [M][ld_z]: pre-activation for GELU'
    int ld_z;
    unsigned* err;
};

// Phi(-|z|) = erfc(|z| / sqrt 2) / 2, the standard normal lower tail, by
// formula 7.1.26 of Abramowitz and Stegun, "Handbook of Mathematical
// Functions": erfc x = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
// t = 1 / (1 + p x), x >= 0, absolute error <= 1.5e-7 (here with x =
// |z| / sqrt 2: p / sqrt 2 and a_k / 2 folded into the constants).
// Evaluated in float32 with the hardware reciprocal and exponential
// approximations, which add a few 1e-7: far below the BF16 rounding of the
// activations (2^-9 relative).  The GELU epilogue bounds the fused forward
// pass; this form takes about half the instructions of the library erff.
// Also returns exp(-z^2 / 2) for the derivative.
__device__ __forceinline__ float phi_lower(float z, float* gauss)
{
    const float az = fabsf(z);
    const float t = __fdividef(1.0f, fmaf(0.23164190f, az, 1.0f));  // p / sqrt 2 = 0.3275911 / 1.41421356
    float poly = fmaf(t, 0.5307027145f, -0.7265760135f);            // a_k / 2
    poly = fmaf(t, poly, 0.7107068705f);
    poly = fmaf(t, poly, -0.142248368f);
    poly = fmaf(t, poly, 0.127414796f);
    poly *= t;
    const float e = __expf(-0.5f * z * z);
    *gauss = e;
    return poly * e;
}

// GELU(z) = z Phi(z) and its derivative Phi(z) + z phi(z), phi the standard
// normal density, with Phi(z) = 1 - Phi(-z) for z >= 0.
__device__ __forceinline__ float gelu_f(float z)
{
    float e;
    const float lt = phi_lower(z, &e);
    return z * (z >= 0.0f ? 1.0f - lt : lt);
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    float e;
    const float lt = phi_lower(z, &e);
    return (z >= 0.0f ? 1.0f - lt : lt) + z * e * 0.39894228040143268f;
}

// GELU of two values with the packed FP32x2 instructions (the fused
// forward's epilogue): the same formula as gelu_f, with
// exp(-z^2 / 2) = 2^(-z^2 log2(e) / 2) on the hardware base-2 exponential
// and Phi(z) = 1/2 + sign(z) (1/2 - Phi(-|z|)), the sign bit of z moved onto
// the bracket, so that each step but the reciprocal and the exponential
// works on both values at once.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 gelu2_f(float2 z)
{
    const float2 az = make_float2(fabsf(z.x), fabsf(z.y));
    const float2 d = __ffma2_rn(make_float2(0.23164190f, 0.23164190f), az, make_float2(1.0f, 1.0f));
    const float2 t = make_float2(__fdividef(1.0f, d.x), __fdividef(1.0f, d.y));
    float2 poly = __ffma2_rn(t, make_float2(0.5307027145f, 0.5307027145f), make_float2(-0.7265760135f, -0.7265760135f));
    poly = __ffma2_rn(t, poly, make_float2(0.7107068705f, 0.7107068705f));
    poly = __ffma2_rn(t, poly, make_float2(-0.142248368f, -0.142248368f));
    poly = __ffma2_rn(t, poly, make_float2(0.127414796f, 0.127414796f));
    poly = __fmul2_rn(poly, t);
    // -z^2 log2(e) / 2
    const float2 a = __fmul2_rn(__fmul2_rn(z, make_float2(-0.72134752f, -0.72134752f)), z);
    const float2 e = make_float2(ex2_approx(a.x), ex2_approx(a.y));
    const float2 lt = __fmul2_rn(poly, e);                                              // Phi(-|z|)
    const float2 hb = __ffma2_rn(lt, make_float2(-1.0f, -1.0f), make_float2(0.5f, 0.5f));  // 1/2 - Phi(-|z|)
    const float2 sh = make_float2(__uint_as_float(__float_as_uint(hb.x) ^ (__float_as_uint(z.x) & 0x80000000u)),
                                  __uint_as_float(__float_as_uint(hb.y) ^ (__float_as_uint(z.y) & 0x80000000u)));
    return __fmul2_rn(z, __fadd2_rn(sh, make_float2(0.5f, 0.5f)));
}

__global__ void k_debug_gelu(const float* __restrict__ z, int n, int grad, float* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (grad == 2) {
        out[i] = gelu2_f(make_float2(z[i], 0.0f)).x;
        return;
    }
    out[i] = grad ? gelu_grad_f(z[i]) : gelu_f(z[i]);
}

// Epilogue, in column chunks of EC (32, or NT when NT < 32), through shared
// memory so that every global store is a coalesced row segment:
//   1. each thread (one accumulator row) loads EC columns from TMEM and
//      writes them, plus the bias where the epilogue adds one, to the FP32
//      staging tile F[128][EC + 4];
//   2. the CTA walks F with 4 consecutive columns per thread (EC / 4
//      threads per row): GELU / GELU' (reading the pre-activation as a
//      coalesced float4), BF16 casts and row stores; the BF16 values of the
//      transposed copy go to T[EC][128 + 8];
//   3. the CTA writes T as rows of the transposed output.
template <int NT>
struct EpiShape {
    static constexpr int EC = NT < 32 ? NT : 32;   // columns per chunk
    static constexpr int FLD = EC + 4;               // F row stride (floats)
    static constexpr int TLD = BM + 8;               // T row stride (BF16)
    static constexpr uint32_t BYTES = BM * FLD * 4 + EC * TLD * 2;
};

template <int NT, int EPI>
__device__ __forceinline__ void gemm_epilogue(const GemmEpi& e, uint32_t tmem, int m0, int n0, uint8_t* stage)
{
    using S = EpiShape<NT>;
    constexpr int EC = S::EC, FLD = S::FLD, TLD = S::TLD;
    float* F = reinterpret_cast<float*>(stage);
    __nv_bfloat16* T = reinterpret_cast<__nv_bfloat16*>(stage + BM * FLD * 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r_own = warp * 32 + lane;
    const bool has_t = (EPI == EPI_BIAS_GELU || EPI == EPI_GELU_GRAD) && e.out_t != nullptr;
    constexpr int TPR = EC / 4;          // threads per row in phase 2
    constexpr int RPP = 128 / TPR;       // rows per pass of the CTA
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += EC) {
        // ---- 1: TMEM -> F (row per thread)
#pragma unroll
        for (int h = 0; h < EC; h += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c0 + h), v);
            if (EPI == EPI_BIAS_GELU || EPI == EPI_BIAS) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + h + j;
                    v[j] += n < e.N ? __ldg(e.bias + n) : 0.0f;
                }
            }
            // float4 stores: the 8 lanes of one store phase hit 32 distinct banks
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4*>(F + r_own * FLD + h + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        __syncthreads();
        // ---- 2: coalesced row segments
        const int cq = (threadIdx.x % TPR) * 4;
        const int n = n0 + c0 + cq;
#pragma unroll 1
        for (int r = threadIdx.x / TPR; r < BM; r += RPP) {
            const int row = m0 + r;
            const float4 x = *reinterpret_cast<const float4*>(F + r * FLD + cq);
            if (row >= e.M || n >= e.N) continue;
            if (EPI == EPI_F32) {
                *reinterpret_cast<float4*>(e.out_f32 + (size_t)blockIdx.z * e.split_stride + (size_t)row * e.ld_f32 + n) = x;
            } else if (EPI == EPI_BIAS) {
                *reinterpret_cast<float4*>(e.out_f32 + (size_t)row * e.ld_f32 + n) = x;
            } else {
                float4 o;
                if (EPI == EPI_BIAS_GELU) {
                    if (e.out_f32) *reinterpret_cast<float4*>(e.out_f32 + (size_t)row * e.ld_f32 + n) = x;
                    o = make_float4(gelu_f(x.x), gelu_f(x.y), gelu_f(x.z), gelu_f(x.w));
                } else {  // EPI_GELU_GRAD
                    const float4 z = __ldg(reinterpret_cast<const float4*>(e.zin + (size_t)row * e.ld_z + n));
                    o = make_float4(x.x * gelu_grad_f(z.x), x.y * gelu_grad_f(z.y), x.z * gelu_grad_f(z.z),
                                    x.w * gelu_grad_f(z.w));
                }
                const __nv_bfloat162 lo = __floats2bfloat162_rn(o.x, o.y), hi = __floats2bfloat162_rn(o.z, o.w);
                uint2 pk;
                pk.x = *reinterpret_cast<const unsigned*>(&lo);
                pk.y = *reinterpret_cast<const unsigned*>(&hi);
                *reinterpret_cast<uint2*>(e.out_bf16 + (size_t)row * e.ld_bf16 + n) = pk;
                if (has_t) {
                    T[(cq + 0) * TLD + r] = lo.x;
                    T[(cq + 1) * TLD + r] = lo.y;
                    T[(cq + 2) * TLD + r] = hi.x;
                    T[(cq + 3) * TLD + r] = hi.y;
                }
            }
        }
        if (has_t) {
            __syncthreads();
            // ---- 3: transposed rows out_t[n][m0 .. m0+127], 8 BF16 per store
#pragma unroll 1
            for (int t = threadIdx.x; t < EC * (BM / 8); t += 128) {
                const int c = t / (BM / 8), r8 = (t % (BM / 8)) * 8;
                const int nn = n0 + c0 + c, row = m0 + r8;
                if (nn < e.N && row < e.M)
                    *reinterpret_cast<uint4*>(e.out_t + (size_t)nn * e.ld_t + row) =
                        *reinterpret_cast<const uint4*>(T + c * TLD + r8);
            }
        }
        __syncthreads();
    }
}

template <int NT, int STAGES>
struct GemmSmem {
    static constexpr uint32_t A_BYTES = BM * BK * 2;
    static constexpr uint32_t B_BYTES = NT * BK * 2;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr uint32_t TILES = STAGES * STAGE > EpiShape<NT>::BYTES ? STAGES * STAGE : EpiShape<NT>::BYTES;
    static constexpr uint32_t TOTAL = 1024 + TILES + 8 * (2 * STAGES + 1) + 16;
    static constexpr uint32_t TMEM_COLS = NT < 32 ? 32 : NT;
};

// One CTA of 128 threads per (M tile, N tile, K split).  Warp 0 lane 0
// streams the A and B tiles through a STAGES-deep TMA ring, warp 1 lane 0
// issues the tcgen05.mma and frees each stage with tcgen05.commit, and all
// four warps read the 128 x NT FP32 accumulator out of tensor memory (warp
// w owns rows 32w .. 32w+31) for the epilogue.  Every wait is bounded; on a
// timeout the kernel records SPH_DEV_TIMEOUT, lets its own copies land,
// frees its tensor memory and returns.
template <int NT, int EPI, int STAGES>
__global__ void __launch_bounds__(128, 2)
k_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, GemmEpi e)
{
    using L = GemmSmem<NT, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t tiles = (raw + 1023u) & ~1023u;
    const uint32_t bars = tiles + L::TILES;
    auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bars + 8u * (uint32_t)(STAGES + s); };
    const uint32_t done = bars + 8u * (uint32_t)(2 * STAGES);
    const uint32_t tmem_slot = done + 8u;
    uint32_t* tmem_slot_ptr = reinterpret_cast<uint32_t*>(smem_raw + (tmem_slot - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * NT;
    const int kb0 = blockIdx.z * e.kb_per_split;
    const int nk = min(e.kb_per_split, e.kb_total - kb0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(done, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, L::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot_ptr;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int issued = 0;
        bool ok = true;
        for (int i = 0; i < nk; ++i) {
            const int s = i % STAGES;
            if (i >= STAGES && !mbar_wait(empty(s), (uint32_t)((i / STAGES) - 1) & 1u, e.err)) {
                ok = false;
                break;
            }
            const uint32_t a = tiles + (uint32_t)s * L::STAGE;
            mbar_expect_tx(full(s), L::STAGE);
            tma_load_2d(&mapA, full(s), a, (kb0 + i) * BK, m0);
            tma_load_2d(&mapB, full(s), a + L::A_BYTES, (kb0 + i) * BK, n0);
            ++issued;
        }
        if (!ok) {
            // let the copies still in flight land before the CTA goes away
            for (int i = max(0, issued - STAGES); i < issued; ++i)
                mbar_wait(full(i % STAGES), (uint32_t)(i / STAGES) & 1u, e.err);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        constexpr uint32_t idesc = umma_idesc_bf16(BM, NT);
        for (int i = 0; i < nk; ++i) {
            const int s = i % STAGES;
            if (!mbar_wait(full(s), (uint32_t)(i / STAGES) & 1u, e.err)) break;
            tc_fence_after();
            const uint32_t a = tiles + (uint32_t)s * L::STAGE;
            const uint32_t b = a + L::A_BYTES;
#pragma unroll
            for (int k = 0; k < BK / UK; ++k)
                umma_bf16(tmem, sw128_desc(a + k * UK * 2), sw128_desc(b + k * UK * 2), idesc,
                          (uint32_t)((i | k) != 0));
            umma_commit(empty(s));
        }
        umma_commit(done);
    }
    __syncwarp();

    // ---- epilogue (the stage buffers are idle once every MMA completed)
    const bool ok = mbar_wait(done, 0, e.err);
    tc_fence_after();
    // the CTA agrees on ok, so that the barriers inside are reached by all
    if (__syncthreads_and(ok ? 1 : 0))
        gemm_epilogue<NT, EPI>(e, tmem, m0, n0, smem_raw + (tiles - raw));
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, L::TMEM_COLS);
}

// ------------------------------------------------------------ host side

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mutex;

static cudaError_t get_encoder()
{
    std::lock_guard<std::mutex> lock(g_encode_mutex);
    if (g_encode) return cudaSuccess;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return cudaSuccess;
}

// Tensor map of a row-major BF16 matrix [rows][cols] (row stride ld
// elements), boxes of 64 columns x box_rows rows, 128-byte swizzle,
// out-of-range elements read as zero.
static cudaError_t make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows)
{
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t elem[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, elem,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int NT, int EPI>
static cudaError_t launch_gemm_t(const CUtensorMap& ma, const CUtensorMap& mb, const GemmEpi& e, int splits,
                                 cudaStream_t s)
{
    // 128-wide tiles with a short K (the layers): 3 stages (96 KB) so that two
    // CTAs share an SM and one's epilogue overlaps the other's main loop;
    // the weight-gradient products (long K over the batch) keep a deeper ring
    constexpr int STAGES = NT >= 256 ? 4 : (NT >= 128 ? (EPI == EPI_F32 ? 6 : 3) : 6);
    using L = GemmSmem<NT, STAGES>;
    static bool attr = false;
    if (!attr) {
        cudaError_t r = cudaFuncSetAttribute(k_gemm<NT, EPI, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L::TOTAL);
        if (r != cudaSuccess) return r;
        attr = true;
    }
    dim3 grid((e.M + BM - 1) / BM, (e.N + NT - 1) / NT, splits);
    k_gemm<NT, EPI, STAGES><<<grid, 128, L::TOTAL, s>>>(ma, mb, e);
    return cudaGetLastError();
}

// C[M][N] = A[M][K] . B[N][K]^T; A, B row-major BF16 with leading
// dimensions lda, ldb (elements, multiples of 8).  NT chooses the N tile.
static cudaError_t gemm(int NT, int EPI, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M,
                        int N, int K, int splits, GemmEpi e, cudaStream_t s, long long* launches)
{
    CUtensorMap ma, mb;
    cudaError_t r = make_map(&ma, A, M, K, lda, BM);
    if (r != cudaSuccess) return r;
    r = make_map(&mb, B, N, K, ldb, NT);
    if (r != cudaSuccess) return r;
    e.M = M;
    e.N = N;
    e.kb_total = (K + BK - 1) / BK;
    splits = splits < 1 ? 1 : (splits > e.kb_total ? e.kb_total : splits);
    e.kb_per_split = (e.kb_total + splits - 1) / splits;
    splits = (e.kb_total + e.kb_per_split - 1) / e.kb_per_split;
    ++*launches;
#define SPH_GEMM_CASE(nt, epi) \
    if (NT == nt && EPI == epi) return launch_gemm_t<nt, epi>(ma, mb, e, splits, s);
    SPH_GEMM_CASE(128, EPI_BIAS_GELU)
    SPH_GEMM_CASE(16, EPI_BIAS)
    SPH_GEMM_CASE(128, EPI_GELU_GRAD)
    SPH_GEMM_CASE(128, EPI_F32)
    SPH_GEMM_CASE(16, EPI_F32)
    SPH_GEMM_CASE(256, EPI_F32)
#undef SPH_GEMM_CASE
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------- MLP kernels

constexpr int MLP_IN = SPH_MLP_IN, MLP_H = SPH_MLP_HIDDEN, MLP_OUT = SPH_MLP_OUT;

// Offsets of the packed parameter vector: W1 b1 W2 b2 W3 b3 W4 b4.
struct ParamLayout {
    int w[4], b[4], wn[4], in[4], out[4];
    __host__ __device__ ParamLayout()
    {
        const int ins[4] = {MLP_IN, MLP_H, MLP_H, MLP_H}, outs[4] = {MLP_H, MLP_H, MLP_H, MLP_OUT};
        int o = 0;
        for (int l = 0; l < 4; ++l) {
            in[l] = ins[l];
            out[l] = outs[l];
            w[l] = o;
            wn[l] = ins[l] * outs[l];
            o += wn[l];
            b[l] = o;
            o += outs[l];
        }
    }
};

// fp32 master -> BF16 W [out][in] and W^T [in][out] for every layer.
__global__ void k_cast_weights(const float* __restrict__ P, __nv_bfloat16* __restrict__ W,
                               __nv_bfloat16* __restrict__ WT)
{
    const ParamLayout L;
    const int total = L.b[3] + MLP_OUT;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        for (int l = 0; l < 4; ++l) {
            if (t >= L.w[l] && t < L.w[l] + L.wn[l]) {
                const int r = (t - L.w[l]) / L.in[l], c = (t - L.w[l]) % L.in[l];
                const __nv_bfloat16 v = __float2bfloat16_rn(P[t]);
                W[t] = v;
                WT[L.w[l] + c * L.out[l] + r] = v;
            }
        }
    }
}

// x [B][MLP_IN] -> x^T [MLP_IN][B]
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ x, int rows, int cols, int ld_in,
                                 __nv_bfloat16* __restrict__ xt, int ld_out)
{
    __shared__ __nv_bfloat16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? x[(size_t)r * ld_in + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) xt[(size_t)c * ld_out + r] = tile[threadIdx.x][i];
    }
}

// Upstream gradient of the loss at the output y [B][16] (FP32):
// phase 0: force loss mean over rows of 1/2 |y[:,0:3] - t[:,0:3]|^2;
// phase 1: error-head loss mean of 1/2 (y[:,3] - t[:,3])^2;
// external: dy given (gradient test).  Writes dY and dY^T in BF16 and adds
// the loss to *loss.
__global__ void k_output_grad(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ dy_in,
                              int B, int phase, __nv_bfloat16* __restrict__ dy, __nv_bfloat16* __restrict__ dyt,
                              int ld_t, float* __restrict__ loss)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (r < B) {
        for (int c = 0; c < MLP_OUT; ++c) {
            float g = 0.f;
            if (dy_in) {
                g = dy_in[(size_t)r * MLP_OUT + c];
            } else if ((phase == 0 && c < 3) || (phase == 1 && c == 3)) {
                const float d = y[(size_t)r * MLP_OUT + c] - t[(size_t)r * 4 + c];
                l += 0.5f * d * d;
                g = d / (float)B;
            }
            const __nv_bfloat16 gb = __float2bfloat16_rn(g);
            dy[(size_t)r * MLP_OUT + c] = gb;
            dyt[(size_t)c * ld_t + r] = gb;
        }
    }
    // block reduction of the loss
    __shared__ float red[256];
    red[threadIdx.x] = l;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) atomicAdd(loss, red[0] / (float)B);
}

// Sum of the split-K partials of a weight gradient into G (FP32).
__global__ void k_reduce_splits(const float* __restrict__ part, int splits, long long stride, int n,
                                float* __restrict__ g)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < splits; ++k) s += part[(size_t)k * stride + t];
        g[t] = s;
    }
}

// Bias gradient: column sums of d [B][cols] (BF16), one thread per column.
__global__ void k_col_sums(const __nv_bfloat16* __restrict__ d, int B, int cols, int ld, float* __restrict__ g)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < B; ++r) s += __bfloat162float(d[(size_t)r * ld + c]);
    g[c] = s;
}

// Adam (Kingma & Ba) on the FP32 master parameters [lo, hi).
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ Mo,
                       float* __restrict__ Vo, int lo, int hi, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    for (int t = lo + blockIdx.x * blockDim.x + threadIdx.x; t < hi; t += gridDim.x * blockDim.x) {
        const float g = G[t];
        const float m = b1 * Mo[t] + (1.f - b1) * g;
        const float v = b2 * Vo[t] + (1.f - b2) * g * g;
        Mo[t] = m;
        Vo[t] = v;
        P[t] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// ------------------------------------------------------------- fused forward

// The forward pass of 128-row tiles (inference), one persistent CTA per SM
// with two tiles in flight (slots 0 and 1), so that the tensor cores work
// on one tile while the epilogue works on the other.  Per slot the input
// tile and then each hidden layer's output stay in one shared-memory buffer
// in the layout the tensor cores read (K-major, 64-column tiles of 128-byte
// rows with the 128-byte swizzle that TMA writes): a layer's epilogue
// starts once that layer's MMAs have completed, so it writes its output
// over its input.  Each slot has a 128 x 256 FP32 accumulator in tensor
// memory (columns 256 j ..).  The 17 weight tiles of the four layers stream
// through a two-stage TMA ring, once per tile and layer.  Warp 16 loads,
// warp 17 issues the MMAs, warps 0 .. 15 are the epilogue (warp w reads
// tensor-memory lanes 32 (w % 4) .. and, in each 64-column K tile, the 16
// columns 16 (w / 4) ..): bias, GELU, BF16, written straight into the next
// layer's operand tile; the last layer's 16 columns go to y with their
// bias.  All three take the work items (tile pair, layer, slot) in the
// same order: for each pair of tiles, layer by layer, slot 0 then slot 1,
// so the MMAs of one slot's next layer run during the epilogue of the
// other slot's current layer.  The K order and the epilogue arithmetic are
// those of the per-layer GEMMs that training runs.  Every wait is bounded.
namespace fused {
constexpr int KB_IN = (MLP_IN + BK - 1) / BK;   // 5 K tiles of the input
constexpr int KB_H = MLP_H / BK;                // 4 K tiles of a hidden layer
constexpr uint32_t A_TILE = BM * BK * 2;        // 16 KB: 128 rows x 64 BF16
constexpr uint32_t W_TILE = MLP_H * BK * 2;     // 32 KB: 256 rows x 64 BF16
constexpr uint32_t BUF = KB_IN * A_TILE;        // 80 KB per slot: the input, then each layer's output
constexpr uint32_t RING = 2 * BUF;
constexpr int STAGES = 2;
constexpr uint32_t BARS = RING + STAGES * W_TILE;
// barriers: full[2], empty[2], then per slot x_full, buf_free, acc_full,
// epi_done; then the TMEM slot
constexpr uint32_t TOTAL = 1024 + BARS + 8 * 12 + 16;
constexpr int EPI_WARPS = 16;
constexpr int LOAD_WARP = EPI_WARPS, MMA_WARP = EPI_WARPS + 1;
constexpr int THREADS = 32 * (EPI_WARPS + 2);
constexpr int EPI_THREADS = 32 * EPI_WARPS;
}  // namespace fused

// byte offset of element (r, c) in a K-major 64-column tile with 128-byte swizzle
__device__ __forceinline__ uint32_t sw128_offset(int r, int c)
{
    return (uint32_t)(r * 128 + ((((c * 2) >> 4) ^ (r & 7)) << 4) + ((c * 2) & 15));
}

__global__ void __launch_bounds__(fused::THREADS, 1)
k_mlp_fused(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapW0,
            const __grid_constant__ CUtensorMap mapW1, const __grid_constant__ CUtensorMap mapW2,
            const __grid_constant__ CUtensorMap mapW3, const float* __restrict__ P, int B, float* __restrict__ y,
            unsigned* __restrict__ err)
{
    using namespace fused;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bars = base + BARS;
    auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bars + 16u + 8u * (uint32_t)s; };
    // slot j: its input tile landed; its buffer read by its last layer's
    // MMAs; its accumulator complete; its epilogue done (every epilogue
    // thread arrives: the layer's output written, the accumulator read)
    auto x_full = [&](int j) { return bars + 32u + 32u * (uint32_t)j; };
    auto buf_free = [&](int j) { return bars + 40u + 32u * (uint32_t)j; };
    auto acc_full = [&](int j) { return bars + 48u + 32u * (uint32_t)j; };
    auto epi_done = [&](int j) { return bars + 56u + 32u * (uint32_t)j; };
    const uint32_t tmem_slot = bars + 96;
    uint32_t* tmem_slot_ptr = reinterpret_cast<uint32_t*>(gbase + BARS + 96);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ParamLayout L;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(x_full(j), 1);
            mbar_init(buf_free(j), 1);
            mbar_init(acc_full(j), 1);
            mbar_init(epi_done(j), EPI_THREADS);
        }
        mbar_fence_init();
    }
    if (warp == LOAD_WARP) tmem_alloc(tmem_slot, 2 * MLP_H);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot_ptr;

    // tiles of this CTA: t = blockIdx.x + i gridDim.x, i = 0 .. ntl - 1; tile
    // i sits in slot i & 1 as that slot's (i >> 1)-th tile.  Work item it =
    // 8 p + 2 l + j: pair p, layer l, slot j (tile 2 p + j, skipped past
    // ntl).  Per slot, its barriers complete one phase per tile (x_full,
    // buf_free) or per tile and layer (acc_full, epi_done: parity l & 1),
    // and none can run two phases ahead of its waiter: each next phase
    // needs an action that follows the wait on the current one.
    const int ntiles = (B + BM - 1) / BM;
    const int ntl = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int items = 8 * ((ntl + 1) / 2);
    auto tile_row = [&](int i) { return ((int)blockIdx.x + i * (int)gridDim.x) * BM; };

    if (warp == LOAD_WARP) {
        if (lane == 0) {
            // ---- loads, in work-item order: a slot's input tile before its
            // layer 0 (once the slot's previous tile has left the buffer),
            // then the item's weight tiles
            int g = 0, nx[2] = {0, 0};  // weight tiles, input tiles per slot issued
            bool ok = true;
            for (int it = 0; it < items && ok; ++it) {
                const int p = it >> 3, l = (it >> 1) & 3, j = it & 1, i = 2 * p + j;
                if (i >= ntl) continue;
                if (l == 0) {
                    if (p > 0 && !mbar_wait(buf_free(j), (uint32_t)(p - 1) & 1u, err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(x_full(j), KB_IN * A_TILE);
                    for (int kb = 0; kb < KB_IN; ++kb)
                        tma_load_2d(&mapX, x_full(j), base + j * BUF + kb * A_TILE, kb * BK, tile_row(i));
                    ++nx[j];
                }
                const CUtensorMap* map = l == 0 ? &mapW0 : l == 1 ? &mapW1 : l == 2 ? &mapW2 : &mapW3;
                const uint32_t bytes = l == 3 ? MLP_OUT * BK * 2 : W_TILE;
                const int nkb = l == 0 ? KB_IN : KB_H;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % STAGES;
                    if (g >= STAGES && !mbar_wait(empty(s), (uint32_t)((g / STAGES) - 1) & 1u, err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(full(s), bytes);
                    tma_load_2d(map, full(s), base + RING + s * W_TILE, kb * BK, 0);
                }
            }
            if (!ok) {  // let the copies in flight land before the CTA goes away
                for (int h = (g > STAGES ? g - STAGES : 0); h < g; ++h)
                    mbar_wait(full(h % STAGES), (uint32_t)(h / STAGES) & 1u, err);
                for (int j = 0; j < 2; ++j)
                    if (nx[j] > 0) mbar_wait(x_full(j), (uint32_t)(nx[j] - 1) & 1u, err);
            }
        }
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            // ---- MMA issue, in work-item order: layer l of a slot once the
            // slot's input tile has landed (l = 0) or once its epilogue of
            // layer l - 1 (of the previous tile for l = 0) is done
            bool ok = true;
            int g = 0;
            for (int it = 0; it < items && ok; ++it) {
                const int p = it >> 3, l = (it >> 1) & 3, j = it & 1, i = 2 * p + j;
                if (i >= ntl) continue;
                if (l == 0) {
                    ok = mbar_wait(x_full(j), (uint32_t)p & 1u, err);
                    if (ok && p > 0) ok = mbar_wait(epi_done(j), 1u, err);  // layer 3 of the slot's previous tile
                } else {
                    ok = mbar_wait(epi_done(j), (uint32_t)(l - 1) & 1u, err);
                }
                if (!ok) break;
                tc_fence_after();
                const uint32_t a_buf = base + j * BUF;
                const uint32_t d_tmem = tmem + (uint32_t)(j * MLP_H);
                const int nkb = l == 0 ? KB_IN : KB_H;
                const uint32_t idesc = umma_idesc_bf16(BM, l == 3 ? MLP_OUT : MLP_H);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % STAGES;
                    if (!mbar_wait(full(s), (uint32_t)(g / STAGES) & 1u, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = a_buf + kb * A_TILE;
                    const uint32_t b = base + RING + s * W_TILE;
#pragma unroll
                    for (int k = 0; k < BK / UK; ++k)
                        umma_bf16(d_tmem, sw128_desc(a + k * UK * 2), sw128_desc(b + k * UK * 2), idesc,
                                  (uint32_t)((kb | k) != 0));
                    umma_commit(empty(s));
                }
                if (!ok) break;
                if (l == 3) umma_commit(buf_free(j));  // the slot's buffer is free once these MMAs are done
                umma_commit(acc_full(j));
            }
            if (!ok) {  // so that the epilogue does not wait for nothing
                umma_commit(acc_full(0));
                umma_commit(acc_full(1));
            }
        }
    } else {
        // ---- epilogue warps, in work-item order
        const int q = warp & 3, part = warp >> 2;
        const int r = q * 32 + lane;  // tile row of this thread
        for (int it = 0; it < items; ++it) {
            const int p = it >> 3, l = (it >> 1) & 3, j = it & 1, i = 2 * p + j;
            if (i >= ntl) continue;
            const bool ok = mbar_wait(acc_full(j), (uint32_t)l & 1u, err);
            tc_fence_after();
            if (!ok) break;
            const float* bias = P + L.b[l];
            const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(j * MLP_H);
            if (l < 3) {
                uint8_t* out = gbase + j * BUF;
                // columns c0 .. c0+15 from the registers of their load: bias
                // (four 16-byte loads), GELU, BF16, then K tile c0 / 64 as two
                // 16-byte chunks
                auto emit = [&](const uint32_t (&rv)[16], int c0) {
                    const float4* b4 = reinterpret_cast<const float4*>(bias + c0);
                    float bb[16];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float4 t = __ldg(b4 + e);
                        bb[4 * e] = t.x;
                        bb[4 * e + 1] = t.y;
                        bb[4 * e + 2] = t.z;
                        bb[4 * e + 3] = t.w;
                    }
                    uint32_t pk[8];
#pragma unroll
                    for (int e = 0; e < 16; e += 2) {
                        const float2 gv = gelu2_f(__fadd2_rn(make_float2(__uint_as_float(rv[e]), __uint_as_float(rv[e + 1])),
                                                             make_float2(bb[e], bb[e + 1])));
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(gv.x, gv.y);
                        pk[e >> 1] = *reinterpret_cast<const uint32_t*>(&h2);
                    }
                    uint8_t* tile = out + (c0 / BK) * A_TILE;
                    const int cc = c0 % BK;
                    *reinterpret_cast<uint4*>(tile + sw128_offset(r, cc)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *reinterpret_cast<uint4*>(tile + sw128_offset(r, cc + 8)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                };
                // warp part p takes columns 64 kt + 16 p .. + 15 of each K
                // tile kt; the next chunk's accumulator load runs while this
                // chunk is worked on
                auto col = [&](int kt) { return kt * BK + part * 16; };
                uint32_t ra[16], rb[16];
                tmem_ld16_async(tb + (uint32_t)col(0), ra);
                tmem_wait16(ra);
#pragma unroll
                for (int kt = 0; kt < KB_H; kt += 2) {
                    tmem_ld16_async(tb + (uint32_t)col(kt + 1), rb);
                    emit(ra, col(kt));
                    tmem_wait16(rb);
                    if (kt + 2 < KB_H) tmem_ld16_async(tb + (uint32_t)col(kt + 2), ra);
                    emit(rb, col(kt + 1));
                    if (kt + 2 < KB_H) tmem_wait16(ra);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            } else if (part == 0) {
                float v[16];
                tmem_ld16(tb, v);
                const int row = tile_row(i) + r;
                if (row < B) {
                    float4* o = reinterpret_cast<float4*>(y + (size_t)row * MLP_OUT);
#pragma unroll
                    for (int e = 0; e < 16; e += 4)
                        o[e / 4] = make_float4(v[e] + __ldg(bias + e), v[e + 1] + __ldg(bias + e + 1),
                                               v[e + 2] + __ldg(bias + e + 2), v[e + 3] + __ldg(bias + e + 3));
                }
            }
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(epi_done(j)) : "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == LOAD_WARP) tmem_dealloc(tmem, 2 * MLP_H);
}

}  // namespace sphk

// ------------------------------------------------------------------ API

using namespace sphk;

struct sph_mlp {
    int max_batch;
    float *P, *G, *Mo, *Vo;            // packed parameters, gradients, Adam moments
    __nv_bfloat16 *W, *WT;             // BF16 weights and transposes (packed like P)
    __nv_bfloat16 *XT;                 // [IN][Bmax]
    __nv_bfloat16 *H[3], *HT[3];       // [B][H], [H][B]
    float* Z[3];                       // [B][H]
    float* Y;                          // [B][16]
    __nv_bfloat16 *DY, *DYT;           // [B][16], [16][B]
    __nv_bfloat16 *D[2], *DT[2];       // [B][H], [H][B] (alternating)
    float* part;                       // split-K partials
    float* loss;
    unsigned* err;
    long long step;
    long long launches;
    char msg[512];
};

static const int SPLITS = 8;

static int mfail(sph_mlp* m, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (m) snprintf(m->msg, sizeof(m->msg), "%s", buf);
    sphk::set_handleless_error(buf);
    return code;
}

#define MLP_TRY(m, expr)                                                                           \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return mfail((m), SPH_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                                \
    } while (0)

struct MCarver {
    uintptr_t base, off;
    template <class T>
    T* take(size_t count)
    {
        off = (off + 255) & ~(uintptr_t)255;
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

static size_t mlp_carve(sph_mlp* m, uintptr_t base)
{
    MCarver c{base, 0};
    const size_t P = SPH_MLP_PARAMS, B = (size_t)m->max_batch;
    m->P = c.take<float>(P);
    m->G = c.take<float>(P);
    m->Mo = c.take<float>(P);
    m->Vo = c.take<float>(P);
    m->W = c.take<__nv_bfloat16>(P);
    m->WT = c.take<__nv_bfloat16>(P);
    m->XT = c.take<__nv_bfloat16>((size_t)MLP_IN * B);
    for (int l = 0; l < 3; ++l) {
        m->H[l] = c.take<__nv_bfloat16>((size_t)MLP_H * B);
        m->HT[l] = c.take<__nv_bfloat16>((size_t)MLP_H * B);
        m->Z[l] = c.take<float>((size_t)MLP_H * B);
    }
    m->Y = c.take<float>((size_t)MLP_OUT * B);
    m->DY = c.take<__nv_bfloat16>((size_t)MLP_OUT * B);
    m->DYT = c.take<__nv_bfloat16>((size_t)MLP_OUT * B);
    for (int l = 0; l < 2; ++l) {
        m->D[l] = c.take<__nv_bfloat16>((size_t)MLP_H * B);
        m->DT[l] = c.take<__nv_bfloat16>((size_t)MLP_H * B);
    }
    m->part = c.take<float>((size_t)SPLITS * MLP_H * MLP_IN);
    m->loss = c.take<float>(4);
    m->err = c.take<unsigned>(4);
    return (c.off + 255) & ~(uintptr_t)255;
}

static GemmEpi epi0(sph_mlp* m)
{
    GemmEpi e;
    memset(&e, 0, sizeof(e));
    e.err = m->err;
    return e;
}

// Forward pass of B rows of x (BF16 [B][IN]); keep = 1 also stores the
// pre-activations and the transposed activations for the backward pass.
static int mlp_forward(sph_mlp* m, const __nv_bfloat16* x, int B, float* y, bool keep, cudaStream_t s)
{
    const ParamLayout L;
    const __nv_bfloat16* in = x;
    int ld_in = MLP_IN, k_in = MLP_IN;
    for (int l = 0; l < 3; ++l) {
        GemmEpi e = epi0(m);
        e.bias = m->P + L.b[l];
        e.out_bf16 = m->H[l];
        e.ld_bf16 = MLP_H;
        if (keep) {
            e.out_f32 = m->Z[l];
            e.ld_f32 = MLP_H;
            e.out_t = m->HT[l];
            e.ld_t = m->max_batch;
        }
        MLP_TRY(m, gemm(128, EPI_BIAS_GELU, in, ld_in, m->W + L.w[l], L.in[l], B, MLP_H, k_in, 1, e, s, &m->launches));
        in = m->H[l];
        ld_in = MLP_H;
        k_in = MLP_H;
    }
    GemmEpi e = epi0(m);
    e.bias = m->P + L.b[3];
    e.out_f32 = y;
    e.ld_f32 = MLP_OUT;
    MLP_TRY(m, gemm(16, EPI_BIAS, in, MLP_H, m->W + L.w[3], MLP_H, B, MLP_OUT, MLP_H, 1, e, s, &m->launches));
    return SPH_OK;
}

// Inference: the four layers in one launch (k_mlp_fused), 128-row tiles.
static int mlp_forward_fused(sph_mlp* m, const __nv_bfloat16* x, int B, float* y, cudaStream_t s)
{
    const ParamLayout L;
    CUtensorMap mx, mw[4];
    MLP_TRY(m, make_map(&mx, x, B, MLP_IN, MLP_IN, BM));
    for (int l = 0; l < 4; ++l)
        MLP_TRY(m, make_map(&mw[l], m->W + L.w[l], L.out[l], L.in[l], L.in[l], L.out[l]));
    static bool attr = false;
    static int sms = 0;
    if (!attr) {
        MLP_TRY(m, cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused::TOTAL));
        int dev = 0;
        MLP_TRY(m, cudaGetDevice(&dev));
        MLP_TRY(m, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        attr = true;
    }
    // persistent: one CTA per SM (the kernel takes one), each looping over
    // the 128-row tiles blockIdx.x, blockIdx.x + gridDim.x, ...
    const int tiles = (B + BM - 1) / BM;
    const int grid = tiles < sms ? tiles : sms;
    k_mlp_fused<<<grid, fused::THREADS, fused::TOTAL, s>>>(mx, mw[0], mw[1], mw[2], mw[3], m->P, B, y, m->err);
    ++m->launches;
    MLP_TRY(m, cudaGetLastError());
    return SPH_OK;
}

// Weight and bias gradients of layer l from its output gradient d [B][out]
// (d^T [out][B] given) and its input^T [in][B].
static int layer_grads(sph_mlp* m, int l, const __nv_bfloat16* d, const __nv_bfloat16* dt, int ld_d,
                       const __nv_bfloat16* in_t, int B, cudaStream_t s)
{
    const ParamLayout L;
    const int nout = L.out[l], nin = L.in[l];
    GemmEpi e = epi0(m);
    e.out_f32 = m->part;
    e.ld_f32 = nin;
    e.split_stride = (long long)nout * nin;
    const int NT = nin > 256 ? 128 : 256;
    MLP_TRY(m, gemm(NT, EPI_F32, dt, m->max_batch, in_t, m->max_batch, nout, nin, B, SPLITS, e, s, &m->launches));
    const int kb = (B + BK - 1) / BK, per = (kb + SPLITS - 1) / SPLITS, splits = (kb + per - 1) / per;
    k_reduce_splits<<<120, 256, 0, s>>>(m->part, splits, e.split_stride, nout * nin, m->G + L.w[l]);
    k_col_sums<<<(nout + 127) / 128, 128, 0, s>>>(d, B, nout, ld_d, m->G + L.b[l]);
    m->launches += 2;
    MLP_TRY(m, cudaGetLastError());
    return SPH_OK;
}

// Backward pass from the output gradient (phase 0 / external: every layer;
// phase 1: the output layer only).
static int mlp_backward(sph_mlp* m, int B, bool trunk, cudaStream_t s)
{
    const ParamLayout L;
    int rc = layer_grads(m, 3, m->DY, m->DYT, MLP_OUT, m->HT[2], B, s);
    if (rc != SPH_OK || !trunk) return rc;
    // d3 = (dY . W4) * gelu'(z3)
    const __nv_bfloat16* dprev = m->DY;
    int ld_prev = MLP_OUT, k_prev = MLP_OUT;
    for (int l = 2; l >= 0; --l) {
        const int cur = l & 1;
        GemmEpi e = epi0(m);
        e.zin = m->Z[l];
        e.ld_z = MLP_H;
        e.out_bf16 = m->D[cur];
        e.ld_bf16 = MLP_H;
        e.out_t = m->DT[cur];
        e.ld_t = m->max_batch;
        MLP_TRY(m, gemm(128, EPI_GELU_GRAD, dprev, ld_prev, m->WT + L.w[l + 1], L.out[l + 1], B, MLP_H, k_prev, 1, e,
                        s, &m->launches));
        rc = layer_grads(m, l, m->D[cur], m->DT[cur], MLP_H, l == 0 ? m->XT : m->HT[l - 1], B, s);
        if (rc != SPH_OK) return rc;
        dprev = m->D[cur];
        ld_prev = MLP_H;
        k_prev = MLP_H;
    }
    return SPH_OK;
}

static int check_batch(sph_mlp* m, int B)
{
    if (!m) return mfail(nullptr, SPH_ERR_ARG, "mlp is NULL");
    if (B <= 0 || B > m->max_batch || (B & 127))
        return mfail(m, SPH_ERR_ARG, "batch %d must be a positive multiple of 128 <= %d", B, m->max_batch);
    return SPH_OK;
}

extern "C" {

int sph_mlp_workspace_size(int max_batch, size_t* bytes)
{
    if (!bytes || max_batch <= 0 || (max_batch & 127))
        return mfail(nullptr, SPH_ERR_ARG, "max_batch must be a positive multiple of 128");
    sph_mlp t;
    memset(&t, 0, sizeof(t));
    t.max_batch = max_batch;
    *bytes = mlp_carve(&t, 0);
    return SPH_OK;
}

int sph_mlp_create(int max_batch, void* workspace, size_t ws_bytes, sph_mlp** out)
{
    size_t need = 0;
    int rc = sph_mlp_workspace_size(max_batch, &need);
    if (rc != SPH_OK) return rc;
    if (!out || !workspace || ((uintptr_t)workspace & 255) || ws_bytes < need)
        return mfail(nullptr, SPH_ERR_ARG, "workspace must be 256-byte aligned and >= %zu bytes", need);
    sph_mlp* m = new (std::nothrow) sph_mlp;
    if (!m) return mfail(nullptr, SPH_ERR_ARG, "out of host memory");
    memset(m, 0, sizeof(*m));
    m->max_batch = max_batch;
    mlp_carve(m, (uintptr_t)workspace);
    cudaError_t e = cudaMemset(workspace, 0, need);
    if (e != cudaSuccess) {
        delete m;
        return mfail(nullptr, SPH_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
    }
    *out = m;
    return SPH_OK;
}

void sph_mlp_destroy(sph_mlp* m) { delete m; }

int sph_mlp_set_params(sph_mlp* m, const float* params, void* stream)
{
    if (!m || !params) return mfail(m, SPH_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    MLP_TRY(m, cudaMemcpyAsync(m->P, params, sizeof(float) * SPH_MLP_PARAMS, cudaMemcpyDeviceToDevice, s));
    MLP_TRY(m, cudaMemsetAsync(m->Mo, 0, sizeof(float) * SPH_MLP_PARAMS, s));
    MLP_TRY(m, cudaMemsetAsync(m->Vo, 0, sizeof(float) * SPH_MLP_PARAMS, s));
    k_cast_weights<<<256, 256, 0, s>>>(m->P, m->W, m->WT);
    ++m->launches;
    MLP_TRY(m, cudaGetLastError());
    m->step = 0;
    return SPH_OK;
}

int sph_mlp_get_optimizer_state(sph_mlp* m, float* grads, float* m1, float* m2, long long* step, void* stream)
{
    if (!m || !grads || !m1 || !m2 || !step) return mfail(m, SPH_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(float) * SPH_MLP_PARAMS;
    MLP_TRY(m, cudaMemcpyAsync(grads, m->G, bytes, cudaMemcpyDeviceToDevice, s));
    MLP_TRY(m, cudaMemcpyAsync(m1, m->Mo, bytes, cudaMemcpyDeviceToDevice, s));
    MLP_TRY(m, cudaMemcpyAsync(m2, m->Vo, bytes, cudaMemcpyDeviceToDevice, s));
    *step = m->step;
    return SPH_OK;
}

int sph_mlp_set_optimizer_state(sph_mlp* m, const float* m1, const float* m2, long long step, void* stream)
{
    if (!m || !m1 || !m2) return mfail(m, SPH_ERR_ARG, "NULL argument");
    if (step < 0) return mfail(m, SPH_ERR_ARG, "step must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(float) * SPH_MLP_PARAMS;
    MLP_TRY(m, cudaMemcpyAsync(m->Mo, m1, bytes, cudaMemcpyDeviceToDevice, s));
    MLP_TRY(m, cudaMemcpyAsync(m->Vo, m2, bytes, cudaMemcpyDeviceToDevice, s));
    m->step = step;
    return SPH_OK;
}

int sph_mlp_get_params(sph_mlp* m, float* params, void* stream)
{
    if (!m || !params) return mfail(m, SPH_ERR_ARG, "NULL argument");
    MLP_TRY(m, cudaMemcpyAsync(params, m->P, sizeof(float) * SPH_MLP_PARAMS, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
    return SPH_OK;
}

int sph_mlp_forward(sph_mlp* m, const void* x, int B, float* y, void* stream)
{
    int rc = check_batch(m, B);
    if (rc != SPH_OK) return rc;
    if (!x || !y || ((uintptr_t)x & 15) || ((uintptr_t)y & 15))
        return mfail(m, SPH_ERR_ARG, "x and y must be 16-byte aligned");
    return mlp_forward_fused(m, (const __nv_bfloat16*)x, B, y, (cudaStream_t)stream);
}

int sph_mlp_gradients(sph_mlp* m, const void* x, const float* dy, int B, float* grads, void* stream)
{
    int rc = check_batch(m, B);
    if (rc != SPH_OK) return rc;
    if (!x || !dy || !grads || ((uintptr_t)x & 15)) return mfail(m, SPH_ERR_ARG, "bad pointers");
    cudaStream_t s = (cudaStream_t)stream;
    dim3 tb(32, 8), tg((MLP_IN + 31) / 32, (B + 31) / 32);
    k_transpose_bf16<<<tg, tb, 0, s>>>((const __nv_bfloat16*)x, B, MLP_IN, MLP_IN, m->XT, m->max_batch);
    ++m->launches;
    rc = mlp_forward(m, (const __nv_bfloat16*)x, B, m->Y, true, s);
    if (rc != SPH_OK) return rc;
    k_output_grad<<<(B + 255) / 256, 256, 0, s>>>(m->Y, nullptr, dy, B, 0, m->DY, m->DYT, m->max_batch, nullptr);
    ++m->launches;
    MLP_TRY(m, cudaGetLastError());
    rc = mlp_backward(m, B, true, s);
    if (rc != SPH_OK) return rc;
    MLP_TRY(m, cudaMemcpyAsync(grads, m->G, sizeof(float) * SPH_MLP_PARAMS, cudaMemcpyDeviceToDevice, s));
    return SPH_OK;
}

int sph_mlp_train_step(sph_mlp* m, const void* x, const float* target, int B, int phase, float lr,
                       float* loss_out, void* stream)
{
    int rc = check_batch(m, B);
    if (rc != SPH_OK) return rc;
    if (!x || !target || ((uintptr_t)x & 15)) return mfail(m, SPH_ERR_ARG, "bad pointers");
    if (phase != 0 && phase != 1) return mfail(m, SPH_ERR_ARG, "phase must be 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    const ParamLayout L;
    dim3 tb(32, 8), tg((MLP_IN + 31) / 32, (B + 31) / 32);
    if (phase == 0) {
        k_transpose_bf16<<<tg, tb, 0, s>>>((const __nv_bfloat16*)x, B, MLP_IN, MLP_IN, m->XT, m->max_batch);
        ++m->launches;
    }
    rc = mlp_forward(m, (const __nv_bfloat16*)x, B, m->Y, true, s);
    if (rc != SPH_OK) return rc;
    MLP_TRY(m, cudaMemsetAsync(m->loss, 0, sizeof(float), s));
    k_output_grad<<<(B + 255) / 256, 256, 0, s>>>(m->Y, target, nullptr, B, phase, m->DY, m->DYT, m->max_batch,
                                                  m->loss);
    ++m->launches;
    MLP_TRY(m, cudaGetLastError());
    rc = mlp_backward(m, B, phase == 0, s);
    if (rc != SPH_OK) return rc;
    ++m->step;
    const float b1 = 0.9f, b2 = 0.999f;
    // bias corrections 1 - beta^t in double (in float32 the difference
    // cancels: 1 - 0.999^t loses most of its digits for small t)
    const float c1 = (float)(1.0 - pow((double)b1, (double)m->step));
    const float c2 = (float)(1.0 - pow((double)b2, (double)m->step));
    if (phase == 0) {
        // every parameter except the error-head row 3 of W4 and b4[3]
        k_adam<<<256, 256, 0, s>>>(m->P, m->G, m->Mo, m->Vo, 0, L.w[3] + 3 * MLP_H, lr, b1, b2, 1e-8f, c1, c2);
        k_adam<<<4, 256, 0, s>>>(m->P, m->G, m->Mo, m->Vo, L.w[3] + 4 * MLP_H, L.b[3] + 3, lr, b1, b2, 1e-8f, c1, c2);
        k_adam<<<1, 32, 0, s>>>(m->P, m->G, m->Mo, m->Vo, L.b[3] + 4, L.b[3] + MLP_OUT, lr, b1, b2, 1e-8f, c1, c2);
        m->launches += 3;
    } else {
        k_adam<<<1, 256, 0, s>>>(m->P, m->G, m->Mo, m->Vo, L.w[3] + 3 * MLP_H, L.w[3] + 4 * MLP_H, lr, b1, b2, 1e-8f,
                                 c1, c2);
        k_adam<<<1, 32, 0, s>>>(m->P, m->G, m->Mo, m->Vo, L.b[3] + 3, L.b[3] + 4, lr, b1, b2, 1e-8f, c1, c2);
        m->launches += 2;
    }
    k_cast_weights<<<256, 256, 0, s>>>(m->P, m->W, m->WT);
    ++m->launches;
    MLP_TRY(m, cudaGetLastError());
    if (loss_out) MLP_TRY(m, cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    return SPH_OK;
}

int sph_mlp_status(sph_mlp* m, unsigned* bits, void* stream)
{
    if (!m || !bits) return mfail(m, SPH_ERR_ARG, "NULL argument");
    unsigned v = 0;
    MLP_TRY(m, cudaMemcpyAsync(&v, m->err, sizeof(unsigned), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    MLP_TRY(m, cudaStreamSynchronize((cudaStream_t)stream));
    *bits = v;
    return SPH_OK;
}

long long sph_mlp_launch_count(sph_mlp* m) { return m ? m->launches : 0; }

int sph_debug_gelu(const float* z, int n, int grad, float* out, void* stream)
{
    if (!z || !out || n < 0 || grad < 0 || grad > 2) return mfail(nullptr, SPH_ERR_ARG, "bad GELU arguments");
    if (n == 0) return SPH_OK;
    k_debug_gelu<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(z, n, grad, out);
    MLP_TRY(nullptr, cudaGetLastError());
    return SPH_OK;
}

int sph_debug_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int splits, float* C,
                   unsigned* err, void* stream)
{
    if (!A || !B || !C || !err || M <= 0 || N <= 0 || K <= 0 || (lda & 7) || (ldb & 7) || (N & 3) || splits < 1)
        return mfail(nullptr, SPH_ERR_ARG, "bad GEMM arguments");
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)C & 15))
        return mfail(nullptr, SPH_ERR_ARG, "A, B, C must be 16-byte aligned");
    GemmEpi e;
    memset(&e, 0, sizeof(e));
    e.err = err;
    e.out_f32 = C;
    e.ld_f32 = N;
    e.split_stride = (long long)M * N;
    long long launches = 0;
    const int NT = N <= 16 ? 16 : (N <= 128 ? 128 : 256);
    cudaError_t r = gemm(NT, EPI_F32, (const __nv_bfloat16*)A, lda, (const __nv_bfloat16*)B, ldb, M, N, K, splits,
                         e, (cudaStream_t)stream, &launches);
    if (r != cudaSuccess) return mfail(nullptr, SPH_ERR_CUDA, "GEMM: %s", cudaGetErrorString(r));
    return SPH_OK;
}

}  // extern "C"
