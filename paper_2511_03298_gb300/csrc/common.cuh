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

// Histogram selection for keys whose high 32 bits are an order-preserving
// integer distance.  hist_find locates, among N unique keys, the bin B (of
// HIST_BINS bins of width 1 above the minimum distance; the last bin takes
// everything beyond) that holds the K-th smallest key, with lt = the number
// of keys in lower bins and inB = the keys in bin B.
constexpr int HIST_BINS = 2048;
struct HistSel {
    uint32_t base;
    int B, lt, inB;
};

__device__ __forceinline__ int hist_bin(uint64_t key, uint32_t base) {
    uint32_t d = (uint32_t)(key >> 32) - base;
    return d < (uint32_t)(HIST_BINS - 1) ? (int)d : HIST_BINS - 1;
}

template <class Load>
__device__ void hist_find(Load load, int N, int K, uint32_t* hist, uint32_t* warp_tot, HistSel* hs) {
    __shared__ uint32_t s_min;
    if (threadIdx.x == 0) s_min = 0xffffffffu;
    for (int b = threadIdx.x; b < HIST_BINS; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    uint32_t mn = 0xffffffffu;
    for (int i = threadIdx.x; i < N; i += blockDim.x) mn = min(mn, (uint32_t)(load(i) >> 32));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) atomicMin(&s_min, mn);
    __syncthreads();
    const uint32_t base = s_min;
    for (int i = threadIdx.x; i < N; i += blockDim.x) atomicAdd(&hist[hist_bin(load(i), base)], 1u);
    __syncthreads();
    const int per = HIST_BINS / blockDim.x;  // blockDim.x divides HIST_BINS
    const int b0 = threadIdx.x * per;
    uint32_t local = 0;
    for (int b = b0; b < b0 + per; ++b) local += hist[b];
    const uint32_t excl = block_exclusive_scan(local, warp_tot);
    if (excl < (uint32_t)K && excl + local >= (uint32_t)K) {
        uint32_t c = excl;
        for (int b = b0; b < b0 + per; ++b) {
            if (c + hist[b] >= (uint32_t)K) {
                hs->base = base;
                hs->B = b;
                hs->lt = (int)c;
                hs->inB = (int)hist[b];
                break;
            }
            c += hist[b];
        }
    }
    __syncthreads();
}

// K smallest of N unique distance keys, sorted, into out[0..K) (K <= N).
// Keys of the bins up to B (K plus the ties of bin B) are gathered into buf
// (cap keys, a power of two) and sorted; if they do not fit, the radix
// select above runs instead.
template <class Load>
__device__ void block_select_hist(Load load, int N, int K, uint64_t* out, uint64_t* buf, int cap,
                                  uint32_t* hist, uint32_t* warp_tot) {
    __shared__ HistSel hs;
    __shared__ int s_cnt;
    if (K <= 0) return;
    if (N <= 512 && N <= cap) {
        block_select_smallest(load, N, K, out, buf, cap, hist);
        return;
    }
    hist_find(load, N, K, hist, warp_tot, &hs);
    const int need = hs.lt + hs.inB;
    if (need > cap) {
        block_select_smallest(load, N, K, out, buf, cap, hist);
        return;
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        uint64_t k = load(i);
        if (hist_bin(k, hs.base) <= hs.B) buf[atomicAdd(&s_cnt, 1)] = k;
    }
    __syncthreads();
    const int S = pow2_ceil(need);
    for (int i = need + threadIdx.x; i < S; i += blockDim.x) buf[i] = KEY_NONE;
    __syncthreads();
    block_bitonic_sort(buf, S);
    for (int i = threadIdx.x; i < K; i += blockDim.x) out[i] = buf[i];
    __syncthreads();
}

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

// K smallest of N unique keys held in shared memory (0 < K < N), in no
// particular order: emit(i, key) for i in [0, K).  A histogram of HIST_BINS
// bins of width 2^shift above the smallest distance (shift: the least that
// fits the distance range) finds the bin B of the K-th key; the lt keys of
// lower bins are emitted as found (indices [0, lt)), the keys of bin B are
// sorted and their first K - lt follow.  *kth (shared) receives the K-th
// smallest key.  Returns false, having emitted nothing, if bin B holds more
// than bcap keys (bcap a power of two, bbuf its scratch).  All threads call.
template <class Emit>
__device__ bool block_topk_smem(const uint64_t* keys, int N, int K, Emit emit, uint64_t* bbuf, int bcap,
                                uint32_t* hist, uint32_t* warp_tot, uint64_t* kth) {
    __shared__ uint32_t s_min, s_max;
    __shared__ int s_out, s_nb;
    __shared__ HistSel hs;
    if (threadIdx.x == 0) {
        s_min = 0xffffffffu;
        s_max = 0u;
        s_out = 0;
        s_nb = 0;
    }
    for (int b = threadIdx.x; b < HIST_BINS; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    uint32_t mn = 0xffffffffu, mx = 0u;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const uint32_t d = (uint32_t)(keys[i] >> 32);
        mn = min(mn, d);
        mx = max(mx, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&s_min, mn);
        atomicMax(&s_max, mx);
    }
    __syncthreads();
    const uint32_t base = s_min;
    int shift = 0;
    while (((s_max - base) >> shift) >= (uint32_t)HIST_BINS) ++shift;
    for (int i = threadIdx.x; i < N; i += blockDim.x) atomicAdd(&hist[((uint32_t)(keys[i] >> 32) - base) >> shift], 1u);
    __syncthreads();
    const int per = HIST_BINS / blockDim.x;  // blockDim.x divides HIST_BINS
    const int b0 = threadIdx.x * per;
    uint32_t local = 0;
    for (int b = b0; b < b0 + per; ++b) local += hist[b];
    const uint32_t excl = block_exclusive_scan(local, warp_tot);
    if (excl < (uint32_t)K && excl + local >= (uint32_t)K) {
        uint32_t c = excl;
        for (int b = b0; b < b0 + per; ++b) {
            if (c + hist[b] >= (uint32_t)K) {
                hs.B = b;
                hs.lt = (int)c;
                hs.inB = (int)hist[b];
                break;
            }
            c += hist[b];
        }
    }
    __syncthreads();
    const int B = hs.B, lt = hs.lt, inB = hs.inB;
    if (inB > bcap) return false;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const uint64_t k = keys[i];
        const int b = (int)(((uint32_t)(k >> 32) - base) >> shift);
        if (b < B) emit(atomicAdd(&s_out, 1), k);
        else if (b == B) bbuf[atomicAdd(&s_nb, 1)] = k;
    }
    __syncthreads();
    const int need = K - lt;
    if (inB <= 32) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const uint64_t v = warp_sort_key(lane < inB ? bbuf[lane] : KEY_NONE, lane);
            if (lane < need) emit(lt + lane, v);
            if (lane == need - 1) *kth = v;
        }
    } else {
        const int S = pow2_ceil(inB);
        for (int i = inB + threadIdx.x; i < S; i += blockDim.x) bbuf[i] = KEY_NONE;
        __syncthreads();
        block_bitonic_sort(bbuf, S);
        for (int i = threadIdx.x; i < need; i += blockDim.x) emit(lt + i, bbuf[i]);
        if (threadIdx.x == 0) *kth = bbuf[need - 1];
    }
    __syncthreads();
    return true;
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
void release(Buffer& b);

int num_sms();

}  // namespace ksc
