// Shared device/host helpers of the KScaNN CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/kscann.h"

namespace ksc {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
const char* get_error();

#define KSC_CHECK_ARG(cond, ...)              \
    do {                                      \
        if (!(cond)) {                        \
            ::ksc::set_error(__VA_ARGS__);    \
            return KSC_EINVAL;                \
        }                                     \
    } while (0)

#define KSC_CHECK_STATE(cond, ...)            \
    do {                                      \
        if (!(cond)) {                        \
            ::ksc::set_error(__VA_ARGS__);    \
            return KSC_ESTATE;                \
        }                                     \
    } while (0)

#define KSC_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::ksc::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                             __FILE__, __LINE__);                                       \
            return e_ == cudaErrorMemoryAllocation ? KSC_ENOMEM : KSC_ECUDA;            \
        }                                                                               \
    } while (0)

#define KSC_LAUNCH_CHECK() KSC_CUDA(cudaGetLastError())

#define KSC_TRY(expr)                 \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ != KSC_OK) return rc_; \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------------ keys
// Candidate key: lexicographic (D, id) as one unsigned 64-bit integer.
__host__ __device__ __forceinline__ uint64_t make_key(int32_t D, int32_t id) {
    return ((uint64_t)((uint32_t)D ^ 0x80000000u) << 32) | (uint64_t)(uint32_t)id;
}
// Order-preserving map of a (non-NaN) fp32 value to uint32.
__host__ __device__ __forceinline__ uint32_t ordered_f32(float f) {
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(f);
#else
    memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float unordered_f32(uint32_t u) {
    u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
#ifdef __CUDA_ARCH__
    f = __uint_as_float(u);
#else
    memcpy(&f, &u, 4);
#endif
    return f;
}
constexpr uint64_t KEY_NONE = ~0ull;

// ------------------------------------------------------------------ block sort / select
// Bitonic sort, ascending, of S (power of two) keys in shared memory.
__device__ __forceinline__ void block_bitonic_sort(uint64_t* s, int S) {
    for (int k = 2; k <= S; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < S; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t a = s[i], b = s[ixj];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) { s[i] = b; s[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

__host__ __device__ __forceinline__ int pow2_ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// K smallest of N unique keys produced by load(i), i in [0, N), written sorted
// to out[0..K) (K <= N).  buf: shared buffer of `cap` keys (cap a power of two,
// cap >= K); hist: 256 shared uint32.  Radix select (8-bit digits, most
// significant first) when N > cap, then one bitonic sort of the K survivors.
template <class Load>
__device__ void block_select_smallest(Load load, int N, int K, uint64_t* out, uint64_t* buf, int cap,
                                      uint32_t* hist) {
    __shared__ uint64_t s_prefix, s_mask;
    __shared__ int s_krem, s_cnt;
    if (K <= 0) return;
    if (N <= cap) {
        int S = pow2_ceil(N);
        for (int i = threadIdx.x; i < S; i += blockDim.x) buf[i] = i < N ? load(i) : KEY_NONE;
        __syncthreads();
        block_bitonic_sort(buf, S);
        for (int i = threadIdx.x; i < K; i += blockDim.x) out[i] = buf[i];
        __syncthreads();
        return;
    }
    if (threadIdx.x == 0) { s_prefix = 0; s_mask = 0; s_krem = K; }
    __syncthreads();
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        uint64_t pre = s_prefix, msk = s_mask;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            uint64_t k = load(i);
            if ((k & msk) == pre) atomicAdd(&hist[(k >> shift) & 255], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int krem = s_krem, acc = 0, b = 0;
            for (; b < 256; ++b) {
                if (acc + (int)hist[b] >= krem) break;
                acc += hist[b];
            }
            s_krem = krem - acc;
            s_prefix = pre | ((uint64_t)b << shift);
            s_mask = msk | (255ull << shift);
        }
        __syncthreads();
    }
    // s_prefix is now the K-th smallest key: gather every key <= it.
    uint64_t kth = s_prefix;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        uint64_t k = load(i);
        if (k <= kth) {
            int slot = atomicAdd(&s_cnt, 1);
            if (slot < cap) buf[slot] = k;
        }
    }
    __syncthreads();
    int S = pow2_ceil(K);
    for (int i = s_cnt + threadIdx.x; i < S; i += blockDim.x) buf[i] = KEY_NONE;
    __syncthreads();
    block_bitonic_sort(buf, S);
    for (int i = threadIdx.x; i < K; i += blockDim.x) out[i] = buf[i];
    __syncthreads();
}

// Exclusive prefix sum over the block (blockDim.x a multiple of 32, <= 1024);
// warp_tot: 32 shared uint32.  Returns this thread's exclusive prefix.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t r = x - v + (w > 0 ? warp_tot[w - 1] : 0);
    __syncthreads();
    return r;
}

constexpr int HIST_BINS = 2048;  // bins of the list-ranking select's score histogram

// Ascending bitonic sort of one key per lane across a warp.
__device__ __forceinline__ uint64_t warp_sort_key(uint64_t v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);
            v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
        }
    }
    return v;
}

// K smallest (0 < K < N) of N unique 64-bit keys given by load(i), by one
// warp, in no particular order: emit(i, key) for i in [0, K); returns the K-th
// smallest.  Radix refinement: a histogram of 256 bins of width 2^shift over
// the undecided key range [lo, hi] (shift: the least that fits) locates the
// bin of the K-th key; the keys of lower bins are emitted and the range
// narrows to that bin, until it holds at most 32 keys, which are sorted across
// the warp.  Keys are unique, so a range of fewer than 256 keys ends it.
// hist: 256 words and bb: 32 keys of the warp's own shared memory.  All 32
// lanes call.
// Each pass reads TOPK_U keys per lane before using them, so that that many
// loads per lane are in flight (the keys usually come from global memory).
constexpr int TOPK_U = 8;

template <class Load, class Emit>
__device__ uint64_t warp_topk(Load load, int N, int K, Emit emit, uint32_t* hist, uint64_t* bb) {
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    uint64_t lo = KEY_NONE, hi = 0ull;
    for (int i0 = 0; i0 < N; i0 += 32 * TOPK_U) {
        uint64_t k[TOPK_U];
#pragma unroll
        for (int u = 0; u < TOPK_U; ++u) {
            const int i = i0 + 32 * u + lane;
            k[u] = i < N ? load(i) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < TOPK_U; ++u) {
            if (i0 + 32 * u + lane < N) {
                lo = k[u] < lo ? k[u] : lo;
                hi = k[u] > hi ? k[u] : hi;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    int out = 0, need = K;
    while (true) {
        int shift = 0;
        while (((hi - lo) >> shift) >= 256ull) ++shift;
        for (int b = lane; b < 256; b += 32) hist[b] = 0u;
        __syncwarp();
        for (int i0 = 0; i0 < N; i0 += 32 * TOPK_U) {
            uint64_t k[TOPK_U];
#pragma unroll
            for (int u = 0; u < TOPK_U; ++u) {
                const int i = i0 + 32 * u + lane;
                k[u] = i < N ? load(i) : KEY_NONE;
            }
#pragma unroll
            for (int u = 0; u < TOPK_U; ++u)
                if (i0 + 32 * u + lane < N && k[u] >= lo && k[u] <= hi)
                    atomicAdd(&hist[(uint32_t)((k[u] - lo) >> shift)], 1u);
        }
        __syncwarp();
        uint32_t c[8], local = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            c[j] = hist[8 * lane + j];
            local += c[j];
        }
        uint32_t incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - local;
        int B = -1, lt = 0, inB = 0;
        if (excl < (uint32_t)need && (uint32_t)need <= incl) {
            uint32_t acc = excl;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (B < 0 && acc + c[j] >= (uint32_t)need) {
                    B = 8 * lane + j;
                    lt = (int)acc;
                    inB = (int)c[j];
                }
                acc += c[j];
            }
        }
        const int owner = __ffs(__ballot_sync(0xffffffffu, B >= 0)) - 1;
        B = __shfl_sync(0xffffffffu, B, owner);
        lt = __shfl_sync(0xffffffffu, lt, owner);  // keys of the range below bin B
        inB = __shfl_sync(0xffffffffu, inB, owner);
        const uint64_t blo = lo + ((uint64_t)B << shift);
        const uint64_t bhi = (hi - blo < (1ull << shift)) ? hi : blo + ((1ull << shift) - 1ull);
        const bool last = inB <= 32;
        int nb = 0;
        for (int i0 = 0; i0 < N; i0 += 32 * TOPK_U) {
            uint64_t k[TOPK_U];
#pragma unroll
            for (int u = 0; u < TOPK_U; ++u) {
                const int i = i0 + 32 * u + lane;
                k[u] = i < N ? load(i) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < TOPK_U; ++u) {
                const int i = i0 + 32 * u + lane;
                const bool e = i < N && k[u] >= lo && k[u] < blo;
                const bool g = last && i < N && k[u] >= blo && k[u] <= bhi;
                const uint32_t me = __ballot_sync(0xffffffffu, e), mg = __ballot_sync(0xffffffffu, g);
                if (e) emit(out + __popc(me & below), k[u]);
                if (g) bb[nb + __popc(mg & below)] = k[u];
                out += __popc(me);
                nb += __popc(mg);
            }
        }
        need -= lt;
        if (last) {
            __syncwarp();
            const uint64_t v = warp_sort_key(lane < inB ? bb[lane] : KEY_NONE, lane);
            if (lane < need) emit(out + lane, v);
            const uint64_t kth = __shfl_sync(0xffffffffu, v, need - 1);
            __syncwarp();
            return kth;
        }
        lo = blo;
        hi = bhi;
        __syncwarp();
    }
}

// The same radix refinement by a whole CTA (blockDim.x a multiple of 32):
// block-wide range, histogram and emission (positions from a shared counter,
// so in no particular order), the bin search and the final sort of at most 32
// keys by warp 0.  For queries with many keys.  All threads call; every
// thread gets the K-th smallest.
template <class Load, class Emit>
__device__ uint64_t block_topk(Load load, int N, int K, Emit emit, uint32_t* hist, uint64_t* bb) {
    __shared__ unsigned long long s_lo, s_hi, s_kth;
    __shared__ int s_B, s_lt, s_inB, s_out, s_nb;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_lo = KEY_NONE;
        s_hi = 0ull;
        s_out = 0;
    }
    __syncthreads();
    uint64_t lo = KEY_NONE, hi = 0ull;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const uint64_t k = load(i);
        lo = k < lo ? k : lo;
        hi = k > hi ? k : hi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    if (lane == 0) {
        atomicMin(&s_lo, (unsigned long long)lo);
        atomicMax(&s_hi, (unsigned long long)hi);
    }
    __syncthreads();
    lo = s_lo;
    hi = s_hi;
    int need = K;
    while (true) {
        int shift = 0;
        while (((hi - lo) >> shift) >= 256ull) ++shift;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
        if (threadIdx.x == 0) s_nb = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const uint64_t k = load(i);
            if (k >= lo && k <= hi) atomicAdd(&hist[(uint32_t)((k - lo) >> shift)], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t c[8], local = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                c[j] = hist[8 * lane + j];
                local += c[j];
            }
            uint32_t incl = local;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - local;
            if (excl < (uint32_t)need && (uint32_t)need <= incl) {
                uint32_t acc = excl;
                int B = -1;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (B < 0 && acc + c[j] >= (uint32_t)need) {
                        B = 8 * lane + j;
                        s_B = B;
                        s_lt = (int)acc;
                        s_inB = (int)c[j];
                    }
                    acc += c[j];
                }
            }
        }
        __syncthreads();
        const int B = s_B, lt = s_lt, inB = s_inB;
        const uint64_t blo = lo + ((uint64_t)B << shift);
        const uint64_t bhi = (hi - blo < (1ull << shift)) ? hi : blo + ((1ull << shift) - 1ull);
        const bool last = inB <= 32;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const uint64_t k = load(i);
            if (k >= lo && k < blo) emit(atomicAdd(&s_out, 1), k);
            else if (last && k >= blo && k <= bhi) bb[atomicAdd(&s_nb, 1)] = k;
        }
        __syncthreads();
        need -= lt;
        if (last) {
            if (threadIdx.x < 32) {
                const uint64_t v = warp_sort_key(lane < inB ? bb[lane] : KEY_NONE, lane);
                if (lane < need) emit(s_out + lane, v);
                if (lane == need - 1) s_kth = v;
            }
            __syncthreads();
            return s_kth;
        }
        lo = blo;
        hi = bhi;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ workspace
// Grow-only device buffers owned by an index (one per role).  Growing
// synchronises the stream before freeing the old buffer.
struct Buffer {
    void* p = nullptr;
    size_t bytes = 0;
};
int ensure(Buffer& b, size_t bytes, cudaStream_t st);
// Count of workspace reallocations so far (captured plans compare it).
unsigned long long workspace_generation();
// Makes captured plans re-capture before their next execution (state they
// baked in, such as a buffer address or a parameter, has changed).
void bump_workspace_generation();
void release(Buffer& b);

int num_sms();

}  // namespace ksc
