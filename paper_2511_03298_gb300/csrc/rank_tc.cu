// Centroid ranking scores (Alg. 2 TopNClusters) on the 5th-generation tensor
// cores: S = Q16 . C16^T (16-bit operands: FP16 when the centroids fit it,
// else BF16) accumulated in FP32 in tensor memory.
//
// One CTA computes a 128 x 256 tile (128 queries x 256 lists): TMA loads the
// K-major BF16 operands into shared memory as 128-byte-swizzled boxes of 64
// elements, one elected thread issues tcgen05.mma (M 128, N 256, K 16 per
// instruction) into a 256-column TMEM accumulator, tcgen05.commit signals an
// mbarrier, and the four warps read their 32 TMEM lanes back with
// tcgen05.ld and write score = ||c||^2 - 2 <q, c> (L2) or -<q, c>.  These
// scores are approximate (16-bit operands); the ranking kernel re-scores in
// FP32 every list that their error bound cannot exclude.
//
// FP8 option (kind::f8f6f4, e4m3 x e4m3, FP32 accumulate): every query and
// centroid row is scaled by a power of two s = 2^(e - 8), e the exponent of
// the row's largest magnitude (so the scaled row peaks in [128, 256), inside
// e4m3's range, and the scaling itself is exact), rounded to e4m3, and the
// accumulated dot product is multiplied back by s_q s_c (exact: a power of
// two).  A 128-element e4m3 box is 128 bytes per row, the same swizzle atom
// as a 64-element 16-bit box, and one MMA takes K = 32, so the tile loop and
// the descriptors are those of the 16-bit path.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "index.cuh"

namespace ksc {

constexpr int TC_M = 128, TC_N = 256, TC_KB = 64;  // tile rows, tile columns, K per TMA box
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;          // bounded mbarrier polls

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Poll an mbarrier phase at most `limit` times; false if it never completed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// Instruction descriptor of kind::f16: A and B both FP16 (fmt 0) or both
// BF16 (fmt 1), K-major, FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_f16kind(int fmt, int M, int N) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// The same with 8-bit operands: kind::f8f6f4, whose instruction descriptor
// gives e4m3 for A and B with format code 0 (so the bits equal those of the
// FP16 descriptor); K = 32 per instruction.
__device__ __forceinline__ void tc_mma_f8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// scores[q][c] for one 128 x 256 tile.  KB = number of K boxes of 128 bytes
// per row (64 16-bit or 128 8-bit elements).  F8: e4m3 operands whose rows
// carry the power-of-two scales qs [nq] and cs [L].
template <bool F8>
__global__ void __launch_bounds__(128, 1) k_rank_gemm_tc(const __grid_constant__ CUtensorMap mapA,
                                                         const __grid_constant__ CUtensorMap mapB, int KB, int64_t nq,
                                                         int L, const float* __restrict__ cn, int spherical,
                                                         int fmt, const float* __restrict__ qs,
                                                         const float* __restrict__ cs, float* __restrict__ scores,
                                                         int32_t* __restrict__ status) {
    constexpr int BOX_K = F8 ? 128 : TC_KB;  // elements per 128-byte box row
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_base;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sA = smem_u32(smem), sB = sA + KB * (TC_M * 128);
    const uint32_t bar_tma = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
    if (threadIdx.x == 0) {
        mbar_init(bar_tma, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool ok = true;
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar_tma, (uint32_t)KB * (TC_M + TC_N) * 128);
        for (int kb = 0; kb < KB; ++kb) {
            tma_load_2d(sA + kb * (TC_M * 128), &mapA, bar_tma, kb * BOX_K, m0);
            tma_load_2d(sB + kb * (TC_N * 128), &mapB, bar_tma, kb * BOX_K, n0);
        }
        ok = mbar_wait(bar_tma, 0, TC_WAIT_LIMIT);
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = idesc_f16kind(fmt, TC_M, TC_N);
            // four MMAs per 128-byte box: K = 16 16-bit or 32 8-bit elements = 32 bytes each
            for (int kb = 0; kb < KB; ++kb)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint64_t a = smem_desc(sA + kb * (TC_M * 128) + k * 32);
                    const uint64_t b = smem_desc(sB + kb * (TC_N * 128) + k * 32);
                    if (F8) tc_mma_f8(tmem, a, b, idesc, (kb | k) != 0);
                    else tc_mma(tmem, a, b, idesc, (kb | k) != 0);
                }
            tc_commit(bar_mma);
        } else {
            atomicOr(status, 2);  // the operand copy never completed: wait (bounded) once more
            mbar_wait(bar_tma, 0, TC_WAIT_LIMIT);
        }
    }
    __syncthreads();
    const bool done = __syncthreads_and(threadIdx.x == 0 ? ok : 1);
    // warp-uniform decision (tcgen05.ld is a warp-collective instruction)
    const bool mma_ok = done && __all_sync(0xffffffffu, mbar_wait(bar_mma, 0, TC_WAIT_LIMIT));
    if (mma_ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // 32 x 32 sub-tiles go through the operand buffers (no longer read: the
        // MMAs have completed) so that each store writes 32 consecutive
        // columns of one row; row stride 33 keeps both sides free of bank conflicts
        float* stage = reinterpret_cast<float*>(smem) + warp * (32 * 33);
        const int64_t qb = (int64_t)m0 + warp * 32;
        for (int c0 = 0; c0 < TC_N; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, r);  // lane = row, r[i] = column c0 + i
#pragma unroll
            for (int i = 0; i < 32; ++i) stage[lane * 33 + i] = __uint_as_float(r[i]);
            __syncwarp();
            const int c = n0 + c0 + lane;
            if (c < L) {
                const float cc = spherical ? 0.f : cn[c];
                const float sc = F8 ? cs[c] : 1.f;
                const int nr = nq - qb < 32 ? (int)(nq - qb) : 32;  // rows of this warp inside the batch
                // sixteen rows at a time: their shared loads, then their stores
#pragma unroll 1
                for (int r0 = 0; r0 < nr; r0 += 16) {
                    float v[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int rr = r0 + u < nr ? r0 + u : nr - 1;
                        // F8: the product of two powers of two, an exact rescaling
                        const float dot = F8 ? stage[rr * 33 + lane] * (qs[qb + rr] * sc) : stage[rr * 33 + lane];
                        v[u] = spherical ? -dot : fmaf(-2.f, dot, cc);
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (r0 + u < nr) scores[(qb + r0 + u) * L + c] = v[u];
                }
            }
            __syncwarp();
        }
    } else if (done && lane == 0) {
        atomicOr(status, 2);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
}

// rows of X (fp32 [n x d]) to 16-bit operands [n x Kp] (FP16 when fp16 is
// set, else BF16; round to nearest), zero-padded K.
__global__ void k_to_16(const float* __restrict__ X, int64_t n, int d, int Kp, int fp16, uint16_t* __restrict__ out) {
    int64_t tot = n * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / Kp;
        int t = (int)(e - r * Kp);
        const float v = t < d ? X[r * d + t] : 0.f;
        out[e] = fp16 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
}

// Per-query bound on |given score - exact score| for every list:
// rel * ||q|| * max||c|| (times 2 for L2, whose score carries -2 <q, c>) plus
// (d + 8) 2^-23 (||q|| + max||c||)^2 for the FP32 rounding of ||c||^2 and of
// the exact FP32 re-score.
//  16-bit tensor-core operands: |<q~, c~> - <q, c>| <= (2u + u^2) sum |q_t c_t|
//    + FP32 accumulation, u = 2^-11 (FP16) or 2^-8 (BF16), and
//    sum |q_t c_t| <= ||q|| ||c|| (Cauchy-Schwarz); for FP16 also the
//    subnormal range's absolute error, 2^-25 per element.  FP16 is used when every
//    centroid element is below 2^14 and a query element above 6e4 voids the
//    bound (err = inf: every list is re-scored).
//  FP32 CUDA cores: a dot product of d terms errs by at most about d 2^-24
//    of sum |q_t c_t|.
__global__ void k_score_err(const float* __restrict__ Q, int64_t nq, int d, float cmax, int spherical, float rel,
                            float qmax, float* __restrict__ err) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nq) return;
    float s = 0.f, mx = 0.f;
    for (int t = 0; t < d; ++t) {
        s = fmaf(Q[q * d + t], Q[q * d + t], s);
        mx = fmaxf(mx, fabsf(Q[q * d + t]));
    }
    if (mx > qmax) {  // an element the 16-bit operand cannot hold: no bound
        err[q] = INFINITY;
        return;
    }
    const float qn = sqrtf(s);
    const float e = rel * qn * cmax * 1.0001f;
    // plus the FP32 rounding of ||c||^2 and of the exact re-score itself
    const float r = (float)(d + 8) * 1.2e-7f * (qn + cmax) * (qn + cmax);
    err[q] = (spherical ? e : 2.f * e) + r;
}

// Queries to 16-bit operands [nq x Kp] (zero-padded K) and, in the same pass,
// the per-query bound of k_score_err.  One warp per query (coalesced rows).
__global__ void k_q16_err(const float* __restrict__ Q, int64_t nq, int d, int Kp, int fp16, float cmax,
                          int spherical, float rel, float qmax, uint16_t* __restrict__ out,
                          float* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nq) return;
    float s = 0.f, mx = 0.f;
    for (int t = lane; t < Kp; t += 32) {
        const float v = t < d ? Q[q * d + t] : 0.f;
        s = fmaf(v, v, s);
        mx = fmaxf(mx, fabsf(v));
        out[q * Kp + t] = fp16 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane != 0) return;
    if (mx > qmax) {  // an element the 16-bit operand cannot hold: no bound
        err[q] = INFINITY;
        return;
    }
    const float qn = sqrtf(s);
    // FP16 elements below 2^-14 are subnormal: their rounding error is up to
    // half the spacing 2^-24 rather than relative, for the query's and the
    // centroids' elements alike: eta sum(|c_t| + |q_t|) <= eta sqrt(d) (|q| +
    // max|c|) (BF16 keeps the FP32 exponent range: its 2^-134 is far below r)
    const float sub = fp16 ? 0x1p-25f * sqrtf((float)d) * (qn + cmax) * 1.01f : 0.f;
    const float e = (rel * qn * cmax + sub) * 1.0001f;
    const float r = (float)(d + 8) * 1.2e-7f * (qn + cmax) * (qn + cmax);
    err[q] = (spherical ? e : 2.f * e) + r;
}

// Power-of-two scale of a row whose largest magnitude is mx: 2^(e - 8) with
// mx = m 2^e, m in [0.5, 1), so mx / s = 256 m lies in [128, 256); 1 for a
// zero row.
__device__ __forceinline__ float f8_row_scale(float mx) {
    if (!(mx > 0.f)) return 1.f;
    int e;
    frexpf(mx, &e);
    return ldexpf(1.f, e - 8);
}

__device__ __forceinline__ uint8_t to_e4m3(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// Rows of X [n x d] to e4m3 [n x Kp] (zero-padded K) with their power-of-two
// scales [n].  One warp per row.
__global__ void k_rows_f8(const float* __restrict__ X, int64_t n, int d, int Kp, uint8_t* __restrict__ out,
                          float* __restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    float mx = 0.f;
    for (int t = lane; t < d; t += 32) mx = fmaxf(mx, fabsf(X[r * d + t]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float s = f8_row_scale(mx);
    const float inv = 1.f / s;  // a power of two: exact
    for (int t = lane; t < Kp; t += 32) out[r * Kp + t] = t < d ? to_e4m3(X[r * d + t] * inv) : (uint8_t)0;
    if (lane == 0) scale[r] = s;
}

// Queries to e4m3 rows [nq x Kp] with their scales and, in the same pass, the
// per-query bound of the FP8 scores (rel from fp8_rel below).
__global__ void k_q8_err(const float* __restrict__ Q, int64_t nq, int d, int Kp, float cmax, int spherical,
                         float rel, uint8_t* __restrict__ out, float* __restrict__ qs, float* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nq) return;
    float s = 0.f, mx = 0.f;
    for (int t = lane; t < d; t += 32) {
        const float v = Q[q * d + t];
        s = fmaf(v, v, s);
        mx = fmaxf(mx, fabsf(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const float sq = f8_row_scale(mx);
    const float inv = 1.f / sq;
    for (int t = lane; t < Kp; t += 32) out[q * Kp + t] = t < d ? to_e4m3(Q[q * d + t] * inv) : (uint8_t)0;
    if (lane != 0) return;
    qs[q] = sq;
    const float qn = sqrtf(s);
    const float e = rel * qn * cmax * 1.0001f;
    const float r = (float)(d + 8) * 1.2e-7f * (qn + cmax) * (qn + cmax);
    err[q] = (spherical ? e : 2.f * e) + r;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// elem: 2 (fp16 selects FP16 or BF16) or 1 (e4m3 bytes); boxes of 128 bytes per row
static int make_map(CUtensorMap* map, const void* base, int64_t rows, int Kp, int box_rows, bool fp16,
                    int elem = 2) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available");
        return KSC_ECUDA;
    }
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * elem};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = elem == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                             : (fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return KSC_ECUDA;
    }
    return KSC_OK;
}

bool tc_rank_supported(const ksc_index* ix) { return ix->d <= 256; }

// Approximate scores [nq x L] with the tensor cores plus the per-query error
// bound err [nq]; the caller re-scores exactly what the bound cannot exclude.
static int err_params(ksc_index* ix, bool tensor_cores, float* rel, float* qmax, cudaStream_t st);

int rank_scores_tc(ksc_index* ix, const float* Q, int64_t nq, float* scores, float* err, cudaStream_t st) {
    const int Kp = (ix->d + TC_KB - 1) / TC_KB * TC_KB;
    const int KB = Kp / TC_KB;
    if (!ix->c_rank_bf16) {
        // operand type: FP16 (11-bit significand) when the centroids fit it
        std::vector<float> ch((size_t)ix->L * ix->d);
        KSC_CUDA(cudaMemcpy(ch.data(), ix->c_rank, sizeof(float) * ch.size(), cudaMemcpyDeviceToHost));
        float mx = 0.f;
        for (float v : ch) mx = fmaxf(mx, fabsf(v));
        ix->tc_fp16 = mx < 16384.f;
        KSC_CUDA(cudaMalloc(&ix->c_rank_bf16, sizeof(uint16_t) * (size_t)ix->L * Kp));
        k_to_16<<<(unsigned)std::min<int64_t>(((int64_t)ix->L * Kp + 255) / 256, 4096), 256, 0, st>>>(
            ix->c_rank, ix->L, ix->d, Kp, ix->tc_fp16, (uint16_t*)ix->c_rank_bf16);
        KSC_LAUNCH_CHECK();
        KSC_TRY(make_map(reinterpret_cast<CUtensorMap*>(ix->map_c), ix->c_rank_bf16, ix->L, Kp, TC_N, ix->tc_fp16));
    }
    KSC_TRY(ensure(ix->ws_qbf16, sizeof(uint16_t) * (size_t)nq * Kp, st));
    uint16_t* qb = (uint16_t*)ix->ws_qbf16.p;
    float rel, qmax;
    KSC_TRY(err_params(ix, true, &rel, &qmax, st));
    k_q16_err<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(Q, nq, ix->d, Kp, ix->tc_fp16, ix->c_rank_max_norm,
                                                         ix->spherical, rel, qmax, qb, err);
    KSC_LAUNCH_CHECK();
    CUtensorMap mapA;
    KSC_TRY(make_map(&mapA, qb, nq, Kp, TC_M, ix->tc_fp16));
    const size_t smem = (size_t)KB * (TC_M + TC_N) * 128 + 1024;
    KSC_CUDA(cudaFuncSetAttribute(k_rank_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((ix->L + TC_N - 1) / TC_N, (unsigned)((nq + TC_M - 1) / TC_M));
    k_rank_gemm_tc<false><<<grid, 128, smem, st>>>(mapA, *reinterpret_cast<const CUtensorMap*>(ix->map_c), KB, nq,
                                                   ix->L, ix->c_rank_sq, ix->spherical, ix->tc_fp16 ? 0 : 1, nullptr,
                                                   nullptr, scores, ix->status);
    KSC_LAUNCH_CHECK();
    ix->launches += 2;
    return KSC_OK;
}

// Relative bound of the FP8 scores' dot products, per ||q|| max||c||.
//  Rounding of a scaled element y to e4m3: |fl(y) - y| <= 2^-4 |y| + 2^-10
//  (relative 2^-4 in the normal range, half the subnormal spacing 2^-9
//  below it).  With the row scale s <= max|x_t| / 128 <= ||x|| / 128 and
//  sum |x_t| <= sqrt(d) ||x||, the error of <q~, c~> is at most
//  (2 u + u^2) ||q|| ||c|| + 2 (1 + u) 2^-10 sqrt(d) / 128 ||q|| ||c|| plus
//  a d 2^-34 term (u = 2^-4).  Products of two e4m3 values are exact in
//  FP32; the accumulation inside the MMA is taken as no worse than 13 bits
//  of precision per addition (d 2^-13 (1 + u)^2 of sum |q~_t c~_t|; a
//  reading: the accumulator's internal precision is not documented here);
//  the rescaling by s_q s_c is exact.
static float fp8_rel(int d) {
    const float u = 0.0625f;
    return (2.f * u + u * u) + 2.f * (1.f + u) * 9.765625e-4f * sqrtf((float)d) / 128.f +
           (float)d * 1.2207e-4f * (1.f + u) * (1.f + u) + 1e-6f;
}

// The same scores from e4m3 operands with per-row power-of-two scales.
int rank_scores_tc8(ksc_index* ix, const float* Q, int64_t nq, float* scores, float* err, cudaStream_t st) {
    const int Kp = (ix->d + 127) / 128 * 128;
    const int KB = Kp / 128;
    if (!ix->c_rank_f8) {
        KSC_CUDA(cudaMalloc(&ix->c_rank_f8, (size_t)ix->L * Kp));
        KSC_CUDA(cudaMalloc(&ix->c_rank_f8_scale, sizeof(float) * ix->L));
        k_rows_f8<<<(unsigned)((ix->L + 7) / 8), 256, 0, st>>>(ix->c_rank, ix->L, ix->d, Kp,
                                                               (uint8_t*)ix->c_rank_f8, ix->c_rank_f8_scale);
        KSC_LAUNCH_CHECK();
        KSC_TRY(make_map(reinterpret_cast<CUtensorMap*>(ix->map_c8), ix->c_rank_f8, ix->L, Kp, TC_N, false, 1));
    }
    float rel, qmax;
    KSC_TRY(err_params(ix, true, &rel, &qmax, st));  // max ||c||
    // e4m3 rows (a multiple of 128 bytes each), then the row scales
    const size_t rows_bytes = (size_t)nq * Kp;
    KSC_TRY(ensure(ix->ws_qbf16, rows_bytes + sizeof(float) * (size_t)nq, st));
    uint8_t* q8 = (uint8_t*)ix->ws_qbf16.p;
    float* qsc = reinterpret_cast<float*>(q8 + rows_bytes);
    k_q8_err<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(Q, nq, ix->d, Kp, ix->c_rank_max_norm, ix->spherical,
                                                        fp8_rel(ix->d), q8, qsc, err);
    KSC_LAUNCH_CHECK();
    CUtensorMap mapA;
    KSC_TRY(make_map(&mapA, q8, nq, Kp, TC_M, false, 1));
    const size_t smem = (size_t)KB * (TC_M + TC_N) * 128 + 1024;
    KSC_CUDA(cudaFuncSetAttribute(k_rank_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((ix->L + TC_N - 1) / TC_N, (unsigned)((nq + TC_M - 1) / TC_M));
    k_rank_gemm_tc<true><<<grid, 128, smem, st>>>(mapA, *reinterpret_cast<const CUtensorMap*>(ix->map_c8), KB, nq,
                                                  ix->L, ix->c_rank_sq, ix->spherical, 0, qsc, ix->c_rank_f8_scale,
                                                  scores, ix->status);
    KSC_LAUNCH_CHECK();
    ix->launches += 2;
    return KSC_OK;
}

// Constants of the score bound: max ||c|| (once per index), the relative
// rounding of the operand type and the largest representable query element.
static int err_params(ksc_index* ix, bool tensor_cores, float* rel, float* qmax, cudaStream_t st) {
    if (ix->c_rank_max_norm <= 0.f) {
        std::vector<float> cn(ix->L);
        KSC_CUDA(cudaMemcpyAsync(cn.data(), ix->c_rank_sq, sizeof(float) * ix->L, cudaMemcpyDeviceToHost, st));
        KSC_CUDA(cudaStreamSynchronize(st));
        float m = 0.f;
        for (float v : cn) m = v > m ? v : m;
        ix->c_rank_max_norm = m > 0.f ? sqrtf(m) : 1e-30f;
    }
    const float u2 = ix->tc_fp16 ? 9.77e-4f + 1e-6f : 0.0078125f + 6.2e-5f;  // 2u + u^2
    *rel = tensor_cores ? u2 + (float)ix->d * 4.8e-7f : (float)(ix->d + 8) * 1.2e-7f;
    *qmax = (tensor_cores && ix->tc_fp16) ? 6.0e4f : INFINITY;
    return KSC_OK;
}

int score_err(ksc_index* ix, const float* Q, int64_t nq, bool tensor_cores, float* err, cudaStream_t st) {
    float rel, qmax;
    KSC_TRY(err_params(ix, tensor_cores, &rel, &qmax, st));
    k_score_err<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(Q, nq, ix->d, ix->c_rank_max_norm, ix->spherical,
                                                              rel, qmax, err);
    KSC_LAUNCH_CHECK();
    ix->launches++;
    return KSC_OK;
}

}  // namespace ksc
