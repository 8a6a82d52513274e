// Query path of KScaNN (Alg. 2 with the leaf scan of Alg. 3) on sm_103a.
//
//   a1 rank     : scores of every (query, list) + per-query top-P select
//   a2 LUT      : FP32 residual tables (Eq. 1), per-query scale, u8 tables
//                 and per-(query, probe) integer bias (8-bit LUT, Sec. 2.5)
//   threshold   : per-query upper bound of the R-th key from its nearest lists
//   a3 scan     : cluster-major work list of (list, query group, block tile);
//                 16-entry sub-LUTs held in registers, looked up with PRMT,
//                 u16x2 lane sums, cross-lane reduce-scatter
//   a5 select   : R smallest (D, id) keys per query (radix select + bitonic)
//   a6 rerank   : exact FP32 distances of the R candidates, top-k
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "index.cuh"
#include "mlp.cuh"
#include "scan.cuh"

namespace ksc {

constexpr int SEL_CAP = 4096;   // bitonic buffer of the select kernels (>= KSC_MAX_RERANK)

// Shared buffer of the exact select of overflowed queries: 8 R keys (a power
// of two, at least 1024, at most SEL_CAP; it sorts the R best).
static int sel_keys(int Rmax) { return std::min(SEL_CAP, std::max(1024, pow2_ceil(8 * Rmax))); }

// Per-query kernels come in two shapes: a warp per query (many queries: the
// GPU is full of warps) or a CTA per query (few queries: eight warps share
// each one).  The warp shape pays off once the batch fills every SM's warps.
static bool warp_per_query(int64_t nq) { return nq >= 8 * (int64_t)num_sms(); }
constexpr int MAX_NPROBE = 4096;
constexpr int NEAR_KEYS_PER_R = 4;  // keys of the unfiltered first scan: at least 4 R ...
constexpr int NEAR_SHARE_DIV = 16;  // ... and at least 1/16 of the keys the query probes

// ------------------------------------------------------------------ a1: list scores
// score[q][c] = ||c||^2 - 2<q,c> (L2, ||q||^2 dropped) or -<q,c> (spherical).
constexpr int SC_T = 64, SC_K = 32;
__global__ void __launch_bounds__(256) k_list_scores(const float* __restrict__ Q, int64_t nq, int d,
                                                     const float* __restrict__ Cc, const float* __restrict__ cn,
                                                     int L, int spherical, float* __restrict__ scores) {
    __shared__ float qs[SC_K][SC_T + 4];
    __shared__ float cs[SC_K][SC_T + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t q0 = (int64_t)blockIdx.y * SC_T;
    const int c0 = blockIdx.x * SC_T;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < d; k0 += SC_K) {
        for (int e = threadIdx.x; e < SC_T * SC_K; e += 256) {
            int r = e / SC_K, kk = e % SC_K;
            int gk = k0 + kk;
            int64_t gq = q0 + r;
            qs[kk][r] = (gq < nq && gk < d) ? Q[gq * d + gk] : 0.f;
            int gc = c0 + r;
            cs[kk][r] = (gc < L && gk < d) ? Cc[(int64_t)gc * d + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < SC_K; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = qs[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = cs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t q = q0 + ty * 4 + i;
        if (q >= nq) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int c = c0 + tx * 4 + j;
            if (c >= L) continue;
            scores[q * L + c] = spherical ? -acc[i][j] : fmaf(-2.f, acc[i][j], cn[c]);
        }
    }
}

// P_q best lists per query.  `scores` may be approximate (each within err[q]
// of the exact score; err = NULL means exact): a float histogram finds the
// bin of the P-th smallest score, every list whose score can still be among
// the P best (score <= upper edge of that bin + 2 err) is re-scored exactly in
// FP32 (L2: sum_t (q_t - c_t)^2 in the direct form; spherical: -<q, c>), and
// the P best by (exact score, list id) are kept.  If more lists qualify than
// the re-score buffer holds (4 Pmax, at least 1024, at most RS_CAP), every
// list is re-scored when all fit, else those with the lowest given scores.
constexpr int RS_CAP = 4096;     // largest re-score buffer
constexpr int FEAT_K = 32;       // list distances of the predictor's features
constexpr int RS_SMEM_L = 8192;  // score rows up to this length are staged in shared memory
__device__ __forceinline__ float exact_list_score(const float* __restrict__ qs, const float* __restrict__ c, int d,
                                                  int spherical, int lane) {
    float acc = 0.f;
    if ((d & 3) == 0) {
        for (int t = lane * 4; t < d; t += 128) {
            float4 cv = __ldg(reinterpret_cast<const float4*>(c + t));
            float4 qv = *reinterpret_cast<const float4*>(qs + t);
            if (spherical) {
                acc = fmaf(qv.x, cv.x, acc); acc = fmaf(qv.y, cv.y, acc);
                acc = fmaf(qv.z, cv.z, acc); acc = fmaf(qv.w, cv.w, acc);
            } else {
                float e0 = qv.x - cv.x, e1 = qv.y - cv.y, e2 = qv.z - cv.z, e3 = qv.w - cv.w;
                acc = fmaf(e0, e0, acc); acc = fmaf(e1, e1, acc); acc = fmaf(e2, e2, acc); acc = fmaf(e3, e3, acc);
            }
        }
    } else {
        for (int t = lane; t < d; t += 32) {
            float cv = __ldg(c + t);
            if (spherical) acc = fmaf(qs[t], cv, acc);
            else { float e = qs[t] - cv; acc = fmaf(e, e, acc); }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return spherical ? -acc : acc;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_rank_select(const float* __restrict__ scores, const float* __restrict__ err,
                                                     const float* __restrict__ Q, const float* __restrict__ Cc,
                                                     int64_t nq, int d, int L, int spherical,
                                                     const int32_t* __restrict__ nprobe_q, int Pfix, int Pmax,
                                                     int rs_cap, int32_t* __restrict__ probes,
                                                     float* __restrict__ score_out, const int32_t* __restrict__ list) {
    extern __shared__ uint64_t cand[];  // rs_cap keys, then the row's scores when L <= RS_SMEM_L
    __shared__ uint32_t hist[HIST_BINS];
    __shared__ uint32_t warp_tot[32];
    __shared__ __align__(16) float qs[KSC_MAX_DIM];
    __shared__ uint32_t s_mn, s_mx;
    __shared__ int s_cnt, s_B;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // every query, or (list != NULL) the list[0] queries list[1..]
    const int64_t count = list ? list[0] : nq;
    for (int64_t e = blockIdx.x; e < count; e += gridDim.x) {
    const int64_t q = list ? list[1 + e] : e;
    __syncthreads();  // the previous query's shared state is no longer read
    int P = nprobe_q ? nprobe_q[q] : Pfix;
    P = P < 1 ? 1 : (P > Pmax ? Pmax : P);
    const float* s = scores + q * L;
    if (L <= RS_SMEM_L) {
        // the row is read from global memory once
        float* ss = reinterpret_cast<float*>(cand + rs_cap);
        for (int c = threadIdx.x; c < L; c += blockDim.x) ss[c] = s[c];
        s = ss;
    }
    const float e2 = err ? 2.f * err[q] : 0.f;
    for (int t = threadIdx.x; t < d; t += blockDim.x) qs[t] = Q[q * d + t];
    if (threadIdx.x == 0) { s_mn = 0xffffffffu; s_mx = 0u; s_cnt = 0; s_B = -1; }
    for (int b = threadIdx.x; b < HIST_BINS; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    uint32_t mn = 0xffffffffu, mx = 0u;
    for (int c = threadIdx.x; c < L; c += blockDim.x) {
        uint32_t u = ordered_f32(s[c]);
        mn = min(mn, u);
        mx = max(mx, u);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) { atomicMin(&s_mn, mn); atomicMax(&s_mx, mx); }
    __syncthreads();
    const float fmn = unordered_f32(s_mn), fmx = unordered_f32(s_mx);
    const float width = (fmx - fmn) / (float)(HIST_BINS - 1);
    const float inv = width > 0.f ? 1.f / width : 0.f;
    auto bin_of = [&](float v) -> int {
        float f = (v - fmn) * inv;
        return f < (float)(HIST_BINS - 1) ? (int)f : HIST_BINS - 1;
    };
    for (int c = threadIdx.x; c < L; c += blockDim.x) atomicAdd(&hist[bin_of(s[c])], 1u);
    __syncthreads();
    {
        const int per = HIST_BINS / blockDim.x;
        const int b0 = threadIdx.x * per;
        uint32_t local = 0;
        for (int b = b0; b < b0 + per; ++b) local += hist[b];
        const uint32_t excl = block_exclusive_scan(local, warp_tot);
        if (excl < (uint32_t)P && excl + local >= (uint32_t)P) {
            uint32_t acc = excl;
            for (int b = b0; b < b0 + per; ++b) {
                if (acc + hist[b] >= (uint32_t)P) { s_B = b; break; }
                acc += hist[b];
            }
        }
    }
    __syncthreads();
    // every list that can still be among the P best
    const float tau = (s_B >= HIST_BINS - 1) ? INFINITY : fmn + (float)(s_B + 1) * width + e2;
    for (int c = threadIdx.x; c < L; c += blockDim.x) {
        if (s[c] <= tau) {
            int slot = atomicAdd(&s_cnt, 1);
            if (slot < rs_cap) cand[slot] = (uint64_t)(uint32_t)c;
        }
    }
    __syncthreads();
    int n = s_cnt;
    if (n > rs_cap) {
        // degenerate score distribution: re-score every list if they fit,
        // else the rs_cap lists with the lowest given scores
        if (L <= rs_cap) {
            n = L;
            for (int c = threadIdx.x; c < L; c += blockDim.x) cand[c] = (uint64_t)(uint32_t)c;
            __syncthreads();
        } else {
            n = rs_cap;
            auto load = [&](int c) -> uint64_t { return ((uint64_t)ordered_f32(s[c]) << 32) | (uint32_t)c; };
            block_select_smallest(load, L, rs_cap, cand, cand, rs_cap, hist);
            for (int i = threadIdx.x; i < rs_cap; i += blockDim.x) cand[i] &= 0xffffffffull;
            __syncthreads();
        }
    }
    for (int i = w; i < n; i += nw) {
        const int c = (int)(uint32_t)cand[i];
        const float v = exact_list_score(qs, Cc + (int64_t)c * d, d, spherical, lane);
        if (lane == 0) cand[i] = ((uint64_t)ordered_f32(v) << 32) | (uint32_t)c;
    }
    __syncthreads();
    if (n <= 32) {
        if (w == 0) {
            const uint64_t v = warp_sort_key(lane < n ? cand[lane] : KEY_NONE, lane);
            cand[lane] = v;
        }
    } else {
        const int S = pow2_ceil(n);
        for (int i = n + threadIdx.x; i < S; i += blockDim.x) cand[i] = KEY_NONE;
        __syncthreads();
        block_bitonic_sort(cand, S);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < Pmax; r += blockDim.x) {
        if (r < P && r < n) {
            probes[q * Pmax + r] = (int32_t)(cand[r] & 0xffffffffu);
            if (score_out) score_out[q * Pmax + r] = unordered_f32((uint32_t)(cand[r] >> 32));
        } else {
            probes[q * Pmax + r] = -1;
            if (score_out) score_out[q * Pmax + r] = INFINITY;
        }
    }
    }
}

// Warp bitonic sort, ascending, of S (a power of two) keys in shared memory.
__device__ __forceinline__ void warp_bitonic_smem(uint64_t* s, int S, int lane) {
    for (int k = 2; k <= S; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < S; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = s[i], b = s[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ uint32_t warp_sort_u32(uint32_t v, int lane) {  // ascending, one value per lane
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
            v = (((lane & k) == 0) == ((lane & j) == 0)) ? min(o, v) : max(o, v);
        }
    }
    return v;
}

// Ascending sort of a bitonic sequence of one value per lane.
__device__ __forceinline__ uint32_t warp_merge_u32(uint32_t v, int lane) {
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
        v = (lane & j) == 0 ? min(o, v) : max(o, v);
    }
    return v;
}

// The K smallest of N values load(i) (order-preserving u32 images of the
// scores, counted with multiplicity; 0 < K <= 48, K < N), ascending into
// vals[0..K), by one warp.  Each lane keeps the two smallest values it reads
// (i = lane, lane + 32, ...).  The K-th smallest t of those (at most) 64 is
// at least the K-th smallest of all values (they are K of them; with N < 64
// they are all of them), so the values at or below t hold the K smallest:
// they are gathered and sorted.  Two passes over the values and a few warp
// sorts, against the radix refinement's histogram passes.  Returns the number
// gathered (>= K), or -1 if more than 64 (the caller then selects by radix
// refinement; at K 48 of 1024 random scores about 65 values fall at or below
// t).  vals: 64 words of the warp's own shared memory.  All 32 lanes call.
template <class Load>
__device__ int warp_small_kvals(Load load, int N, int K, uint32_t* vals) {
    const int lane = threadIdx.x & 31;
    uint32_t a = 0xffffffffu, b = 0xffffffffu;  // a <= b: the two smallest values of this lane
    for (int i0 = 0; i0 < N; i0 += 32 * TOPK_U) {
        uint32_t x[TOPK_U];
#pragma unroll
        for (int u = 0; u < TOPK_U; ++u) {
            const int i = i0 + 32 * u + lane;
            x[u] = i < N ? load(i) : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < TOPK_U; ++u) {
            b = min(b, max(a, x[u]));
            a = min(a, x[u]);
        }
    }
    // both sets sorted across the warp; against the reversed second, the
    // element-wise minima are the 32 smallest of the 64 and the maxima the
    // 32 largest, each a bitonic sequence
    const uint32_t A = warp_sort_u32(a, lane), B = warp_sort_u32(b, lane);
    const uint32_t Br = __shfl_sync(0xffffffffu, B, 31 - lane);
    const uint32_t v = warp_merge_u32(K <= 32 ? min(A, Br) : max(A, Br), lane);
    const uint32_t t = __shfl_sync(0xffffffffu, v, (K - 1) & 31);
    const uint32_t below = (1u << lane) - 1u;
    int n = 0;
    for (int i0 = 0; i0 < N; i0 += 32) {
        const int i = i0 + lane;
        const uint32_t x = i < N ? load(i) : 0xffffffffu;
        const bool in = i < N && x <= t;
        const uint32_t m = __ballot_sync(0xffffffffu, in);
        const int at = n + __popc(m & below);
        if (in && at < 64) vals[at] = x;
        n += __popc(m);
    }
    if (n > 64) return -1;
    __syncwarp();
    const uint32_t c0 = lane < n ? vals[lane] : 0xffffffffu, c1 = lane + 32 < n ? vals[lane + 32] : 0xffffffffu;
    const uint32_t S0 = warp_sort_u32(c0, lane);
    if (n <= 32) {
        __syncwarp();
        vals[lane] = S0;
    } else {
        const uint32_t S1r = __shfl_sync(0xffffffffu, warp_sort_u32(c1, lane), 31 - lane);
        const uint32_t lo = warp_merge_u32(min(S0, S1r), lane), hi = warp_merge_u32(max(S0, S1r), lane);
        __syncwarp();
        vals[lane] = lo;
        vals[lane + 32] = hi;
    }
    __syncwarp();
    return n;
}

// One warp per query (RSW_WARPS per CTA) for L <= RSW_MAX_L: the row of given
// scores is staged in the warp's shared memory and the P-th smallest given
// score s_P found by radix refinement over (score, list) keys.  Every list of
// the exact top P has a given score <= s_P + 2 err (P lists have given scores
// <= s_P, so the exact P-th score is at most s_P + err).  Those lists are
// re-scored exactly in FP32 (8 at a time, as in the re-rank) and the P best by
// (score, id) are sorted.  A query with more than RSW_CAND such lists is put on
// `redo` for k_rank_select.
constexpr int RSW_WARPS = 4;
constexpr int RSW_MAX_L = 2048;
constexpr int RSW_CAND = 128;

// A row of L scores into the warp's shared memory ss, with up to 8 16-byte
// loads per lane in flight (ss 16-byte aligned).
__device__ __forceinline__ void stage_row(const float* __restrict__ row, float* ss, int L, int lane) {
    if ((L & 3) == 0 && (reinterpret_cast<uintptr_t>(row) & 15) == 0) {
        const float4* r4 = reinterpret_cast<const float4*>(row);
        float4* s4 = reinterpret_cast<float4*>(ss);
        const int L4 = L >> 2;
        for (int c0 = 0; c0 < L4; c0 += 32 * 8) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + 32 * u + lane;
                v[u] = c < L4 ? __ldg(r4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + 32 * u + lane;
                if (c < L4) s4[c] = v[u];
            }
        }
    } else {
        for (int c = lane; c < L; c += 32) ss[c] = row[c];
    }
    __syncwarp();
}

// The lists of given score <= tau (staged in ss) into ck, ascending; returns
// their number (only the first RSW_CAND are stored).  One warp.
__device__ __forceinline__ int collect_lists(const float* ss, int L, float tau, uint64_t* ck, int lane) {
    const uint32_t below = (1u << lane) - 1u;
    int n = 0;
    for (int c0 = 0; c0 < L; c0 += 32) {
        const int c = c0 + lane;
        const bool in = c < L && ss[c] <= tau;
        const uint32_t m = __ballot_sync(0xffffffffu, in);
        const int at = n + __popc(m & below);
        if (in && at < RSW_CAND) ck[at] = (uint64_t)(uint32_t)c;
        n += __popc(m);
    }
    return n;
}

// The n (<= RSW_CAND) lists in ck re-scored exactly in FP32 (8 at a time, as
// in the re-rank), sorted by (score, id); the P best into row q of probes
// (and score_out), -1 (+inf) past them up to Pmax.  One warp.
__device__ void exact_top_p(int64_t q, int n, int P, int Pmax, uint64_t* ck, const float* __restrict__ Q,
                            const float* __restrict__ Cc, int d, int spherical, int32_t* __restrict__ probes,
                            float* __restrict__ score_out, int lane) {
    __syncwarp();
    // exact FP32 scores, 8 lists at a time
    const float* qv = Q + q * d;
    const bool vec = (d & 3) == 0 && d <= 128;
    const int myrow = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    for (int i0 = 0; i0 < n; i0 += 8) {
        float a[8];
        if (vec) {
            const bool inl = lane * 4 < d;
            float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (inl) q4 = make_float4(qv[lane * 4], qv[lane * 4 + 1], qv[lane * 4 + 2], qv[lane * 4 + 3]);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = i0 + u < n ? (int)(uint32_t)ck[i0 + u] : -1;
                const float4 cv = (c >= 0 && inl) ? __ldg(reinterpret_cast<const float4*>(Cc + (int64_t)c * d) + lane)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                if (spherical) {
                    a[u] = fmaf(q4.w, cv.w, fmaf(q4.z, cv.z, fmaf(q4.y, cv.y, q4.x * cv.x)));
                } else {
                    const float e0 = q4.x - cv.x, e1 = q4.y - cv.y, e2 = q4.z - cv.z, e3 = q4.w - cv.w;
                    a[u] = fmaf(e3, e3, fmaf(e2, e2, fmaf(e1, e1, e0 * e0)));
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = i0 + u < n ? (int)(uint32_t)ck[i0 + u] : -1;
                float acc = 0.f;
                if (c >= 0) {
                    for (int t = lane; t < d; t += 32) {
                        const float x = __ldg(Cc + (int64_t)c * d + t);
                        if (spherical) acc = fmaf(qv[t], x, acc);
                        else { const float e = qv[t] - x; acc = fmaf(e, e, acc); }
                    }
                }
                a[u] = acc;
            }
        }
        // halving exchange: lane ends with the sum of row myrow
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool up = lane & 16;
            const float send = up ? a[i] : a[i + 4], keep = up ? a[i + 4] : a[i];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const bool up = lane & 8;
            const float send = up ? a[i] : a[i + 2], keep = up ? a[i + 2] : a[i];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
        {
            const bool up = lane & 4;
            const float send = up ? a[0] : a[1], keep = up ? a[1] : a[0];
            a[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        a[0] += __shfl_xor_sync(0xffffffffu, a[0], 2);
        a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
        __syncwarp();
        const int i = i0 + myrow;
        if ((lane & 3) == 0 && i < n) {
            const uint32_t c = (uint32_t)ck[i];
            ck[i] = ((uint64_t)ordered_f32(spherical ? -a[0] : a[0]) << 32) | c;
        }
        __syncwarp();
    }
    // the P best in order
    if (n <= 32) {
        const uint64_t v = warp_sort_key(lane < n ? ck[lane] : KEY_NONE, lane);
        ck[lane] = v;
    } else {
        const int S = pow2_ceil(n);
        for (int i = n + lane; i < S; i += 32) ck[i] = KEY_NONE;
        __syncwarp();
        warp_bitonic_smem(ck, S, lane);
    }
    __syncwarp();
    for (int r = lane; r < Pmax; r += 32) {
        if (r < P && r < n) {
            probes[q * Pmax + r] = (int32_t)(ck[r] & 0xffffffffu);
            if (score_out) score_out[q * Pmax + r] = unordered_f32((uint32_t)(ck[r] >> 32));
        } else {
            probes[q * Pmax + r] = -1;
            if (score_out) score_out[q * Pmax + r] = INFINITY;
        }
    }
}


__global__ void __launch_bounds__(RSW_WARPS * 32) k_rank_select_w(const float* __restrict__ scores,
                                                                  const float* __restrict__ err,
                                                                  const float* __restrict__ Q,
                                                                  const float* __restrict__ Cc, int64_t nq, int d,
                                                                  int L, int spherical,
                                                                  const int32_t* __restrict__ nprobe_q, int Pfix,
                                                                  int Pmax, int32_t* __restrict__ probes,
                                                                  float* __restrict__ score_out,
                                                                  int32_t* __restrict__ redo,
                                                                  float* __restrict__ feat) {
    extern __shared__ uint64_t rsm[];  // RSW_WARPS x RSW_CAND keys, then RSW_WARPS x L scores
    __shared__ uint32_t hist[RSW_WARPS][256];
    __shared__ uint64_t bb[RSW_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * RSW_WARPS + w;
    if (q >= nq) return;
    uint64_t* ck = rsm + w * RSW_CAND;
    float* ss = reinterpret_cast<float*>(rsm + RSW_WARPS * RSW_CAND) + (size_t)w * L;
    int P = nprobe_q ? nprobe_q[q] : Pfix;
    P = P < 1 ? 1 : (P > Pmax ? Pmax : P);
    stage_row(scores + q * L, ss, L, lane);
    float tau = INFINITY;
    auto load = [&](int c) -> uint64_t { return ((uint64_t)ordered_f32(ss[c]) << 32) | (uint32_t)c; };
    auto load32 = [&](int c) -> uint32_t { return ordered_f32(ss[c]); };
    uint32_t* kv = reinterpret_cast<uint32_t*>(ck);  // the small selection's values (ck's first 64 words)
    if (feat) {
        // the K = max(P, FEAT_K) smallest given scores, sorted: the predictor's
        // distances (+ ||q||^2 for L2, which the score leaves out) and s_P
        const int K = min(max(P, FEAT_K), L);
        uint32_t fv, sP = 0u;  // this lane's distance, the P-th smallest (ordered images)
        if (K < L && K <= 48 && warp_small_kvals(load32, L, K, kv) >= 0) {
            fv = kv[lane];
            if (P < L) sP = kv[P - 1];
        } else {
            auto emit = [&](int i, uint64_t k) { ck[i] = k; };
            if (K < L) warp_topk(load, L, K, emit, hist[w], bb[w]);
            else for (int c = lane; c < L; c += 32) ck[c] = load(c);
            const int S = pow2_ceil(K);
            for (int i = K + lane; i < S; i += 32) ck[i] = KEY_NONE;
            __syncwarp();
            warp_bitonic_smem(ck, S, lane);
            fv = (uint32_t)(ck[lane] >> 32);
            if (P < L) sP = (uint32_t)(ck[P - 1] >> 32);
        }
        float qq = 0.f;
        if (!spherical) {
            for (int t = lane; t < d; t += 32) qq = fmaf(Q[q * d + t], Q[q * d + t], qq);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) qq += __shfl_xor_sync(0xffffffffu, qq, o);
        }
        feat[q * FEAT_K + lane] = unordered_f32(fv) + qq;
        if (P < L) tau = unordered_f32(sP) + (err ? 2.f * err[q] : 0.f);
        __syncwarp();
    } else if (P < L) {
        uint32_t sP;
        if (P <= 48 && warp_small_kvals(load32, L, P, kv) >= 0) {
            sP = kv[P - 1];
            __syncwarp();  // ck is reused for the lists below
        } else {
            auto none = [](int, uint64_t) {};
            sP = (uint32_t)(warp_topk(load, L, P, none, hist[w], bb[w]) >> 32);
        }
        tau = unordered_f32(sP) + (err ? 2.f * err[q] : 0.f);
    }
    // the lists that can still be among the P best
    const int n = collect_lists(ss, L, tau, ck, lane);
    if (n > RSW_CAND) {
        if (lane == 0) redo[1 + atomicAdd(&redo[0], 1)] = (int32_t)q;
        return;
    }
    exact_top_p(q, n, P, Pmax, ck, Q, Cc, d, spherical, probes, score_out, lane);
}

// The adaptive search's ranking in one kernel (Sec. 4.2.1-4.2.2, Eq. 2), a
// warp per query, persistent CTAs of RH_WARPS warps: the FEAT_K smallest
// given scores (the predictor's distances, as k_feat_scores), the features,
// network and settings (as k_features and k_mlp_infer, the same operations
// in the same order: bit for bit their settings), then the exact ranking of
// the predicted nprobe lists (as k_rank_select_w).  The BF16-rounded hidden
// weights are staged once per CTA as BF16 pairs [input f][units 2l, 2l + 1]
// (rows of 33 words: the transposing stores fall in distinct banks; BF16
// keeps the CTA small enough for three per SM), so that lane l accumulates
// units 2l and 2l + 1 from one 4-byte load and one packed FMA per input
// (each half the scalar FMA's result); the inputs are broadcast by shuffles.
// Writes nprobe_out / rerank_out; a query with more than RSW_CAND lists
// inside its bound goes on `redo`.
constexpr int RH_WARPS = 8;
constexpr int RH_WLD = 33;  // words per input row of the staged weight pairs
constexpr size_t rh_head_bytes() { return sizeof(uint32_t) * 2 * MLP_F * RH_WLD + sizeof(float) * (4 * MLP_H + 4); }

// The two BF16 values of a staged pair as FP32 (exact).
__device__ __forceinline__ float2 bf16_pair(uint32_t pk) {
    return make_float2(__uint_as_float(pk << 16), __uint_as_float(pk & 0xffff0000u));
}
constexpr size_t rh_warp_bytes(int L) {
    return sizeof(uint64_t) * (RSW_CAND + 32) + sizeof(uint32_t) * 256 + sizeof(float) * (size_t)((L + 3) & ~3);
}

__global__ void __launch_bounds__(RH_WARPS * 32) k_rank_head_w(const float* __restrict__ scores,
                                                               const float* __restrict__ err,
                                                               const float* __restrict__ Q,
                                                               const float* __restrict__ Cc, int64_t nq, int d, int L,
                                                               int spherical, const float* __restrict__ wm,
                                                               ksc_adaptive_params prm, int Pmax,
                                                               int32_t* __restrict__ probes,
                                                               int32_t* __restrict__ redo,
                                                               int32_t* __restrict__ nprobe_out,
                                                               int32_t* __restrict__ rerank_out) {
    extern __shared__ uint64_t hsm[];
    uint32_t* WB1 = reinterpret_cast<uint32_t*>(hsm);
    uint32_t* WB2 = WB1 + MLP_F * RH_WLD;
    float* hb1 = reinterpret_cast<float*>(WB2 + MLP_H * RH_WLD);
    float* hb2 = hb1 + MLP_H;
    float* hW3 = hb2 + MLP_H;  // [f][o]
    float* hb3 = hW3 + MLP_O * MLP_H;
    unsigned char* wbase = reinterpret_cast<unsigned char*>(hsm) + rh_head_bytes();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char* mine = wbase + (size_t)w * rh_warp_bytes(L);
    uint64_t* ck = reinterpret_cast<uint64_t*>(mine);
    uint64_t* bb = ck + RSW_CAND;
    uint32_t* hist = reinterpret_cast<uint32_t*>(bb + 32);
    float* ss = reinterpret_cast<float*>(hist + 256);
    uint32_t* kv = reinterpret_cast<uint32_t*>(ck);
    {
        // hidden weights: coalesced 16-byte loads of rows a, stored transposed
        // as BF16 (units 2l, 2l + 1 of input f in word f * RH_WLD + l)
        const MlpW G = mlp_views(wm);
        constexpr int V = MLP_H * MLP_F / 4 / (RH_WARPS * 32);
        float4 v1[V], v2[V];
#pragma unroll
        for (int u = 0; u < V; ++u) {
            v1[u] = __ldg(reinterpret_cast<const float4*>(G.W1) + threadIdx.x + RH_WARPS * 32 * u);
            v2[u] = __ldg(reinterpret_cast<const float4*>(G.W2) + threadIdx.x + RH_WARPS * 32 * u);  // (MLP_F == MLP_H)
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int e4 = threadIdx.x + RH_WARPS * 32 * u, a = e4 >> 4, f = 4 * (e4 & 15);
            const float x1[4] = {v1[u].x, v1[u].y, v1[u].z, v1[u].w}, x2[4] = {v2[u].x, v2[u].y, v2[u].z, v2[u].w};
            __nv_bfloat16* B1 = reinterpret_cast<__nv_bfloat16*>(WB1);
            __nv_bfloat16* B2 = reinterpret_cast<__nv_bfloat16*>(WB2);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                B1[2 * (f + k) * RH_WLD + a] = __float2bfloat16_rn(x1[k]);
                B2[2 * (f + k) * RH_WLD + a] = __float2bfloat16_rn(x2[k]);
            }
        }
        for (int e = threadIdx.x; e < MLP_H; e += blockDim.x) {
            hb1[e] = bf(G.b1[e]);
            hb2[e] = bf(G.b2[e]);
        }
        for (int e = threadIdx.x; e < MLP_O * MLP_H; e += blockDim.x) {  // interleaved: [f][o]
            const int o = e / MLP_H, f = e - o * MLP_H;
            hW3[2 * f + o] = bf(G.W3[e]);
        }
        if (threadIdx.x < MLP_O) hb3[threadIdx.x] = bf(G.b3[threadIdx.x]);
    }
    __syncthreads();
    auto load = [&](int c) -> uint64_t { return ((uint64_t)ordered_f32(ss[c]) << 32) | (uint32_t)c; };
    auto load32 = [&](int c) -> uint32_t { return ordered_f32(ss[c]); };
    for (int64_t q = (int64_t)blockIdx.x * RH_WARPS + w; q < nq; q += (int64_t)gridDim.x * RH_WARPS) {
        stage_row(scores + q * L, ss, L, lane);
        // the FEAT_K smallest scores, ascending (order-preserving images)
        uint32_t fv;
        if (L > FEAT_K && warp_small_kvals(load32, L, FEAT_K, kv) >= 0) {
            fv = kv[lane];
        } else {
            auto emit = [&](int i, uint64_t k) { ck[i] = k; };
            if (L > FEAT_K) warp_topk(load, L, FEAT_K, emit, hist, bb);
            else ck[lane] = load(lane);
            __syncwarp();
            fv = (uint32_t)(warp_sort_key(ck[lane], lane) >> 32);
        }
        __syncwarp();
        float qq = 0.f;
        if (!spherical) {
            for (int t = lane; t < d; t += 32) qq = fmaf(Q[q * d + t], Q[q * d + t], qq);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) qq += __shfl_xor_sync(0xffffffffu, qq, o);
        }
        // features: lane i holds d_i / mean and d_1 / d_i (BF16)
        const float u = fmaxf(feat_dist(unordered_f32(fv) + qq, spherical), 0.f);
        float mean = 0.f;
#pragma unroll
        for (int i = 0; i < MLP_FEAT_K; ++i) mean += __shfl_sync(0xffffffffu, u, i);
        mean = mean / MLP_FEAT_K + 1e-12f;
        const float d1 = __shfl_sync(0xffffffffu, u, 0) + 1e-12f, di = u + 1e-12f;
        const float xa = bf(di / mean), xb = bf(d1 / di);
        // hidden layers: lane l computes units 2l and 2l + 1
        float2 acc = *reinterpret_cast<const float2*>(hb1 + 2 * lane);
#pragma unroll 8
        for (int f = 0; f < MLP_F; ++f) {
            const float x = __shfl_sync(0xffffffffu, f < MLP_FEAT_K ? xa : xb, f & 31);
            acc = f2_fma(make_float2(x, x), bf16_pair(WB1[f * RH_WLD + lane]), acc);
        }
        const float h0 = bf(acc.x > 0.f ? acc.x : 0.f), h1 = bf(acc.y > 0.f ? acc.y : 0.f);
        acc = *reinterpret_cast<const float2*>(hb2 + 2 * lane);
#pragma unroll 8
        for (int f = 0; f < MLP_H; ++f) {
            const float x = __shfl_sync(0xffffffffu, (f & 1) ? h1 : h0, f >> 1);
            acc = f2_fma(make_float2(x, x), bf16_pair(WB2[f * RH_WLD + lane]), acc);
        }
        const float g0 = bf(acc.x > 0.f ? acc.x : 0.f), g1 = bf(acc.y > 0.f ? acc.y : 0.f);
        float2 z = make_float2(hb3[0], hb3[1]);
#pragma unroll 8
        for (int f = 0; f < MLP_H; ++f) {
            const float x = __shfl_sync(0xffffffffu, (f & 1) ? g1 : g0, f >> 1);
            z = f2_fma(make_float2(x, x), *reinterpret_cast<const float2*>(hW3 + 2 * f), z);
        }
        const float p0 = 1.f / (1.f + expf(-z.x)), p1 = 1.f / (1.f + expf(-z.y));
        const int np = prm.regression ? regmap(p0, prm.pmin, prm.pmax, prm.p0, prm.p1)
                                      : eq2(p0, prm.pmin, prm.pmax, prm.p0, prm.p1);
        const int rr = prm.regression ? regmap(p1, prm.rmin, prm.rmax, prm.r0, prm.r1)
                                      : eq2(p1, prm.rmin, prm.rmax, prm.r0, prm.r1);
        if (lane == 0) {
            nprobe_out[q] = np;
            rerank_out[q] = rr;
        }
        // the exact ranking of the predicted lists
        const int P = np < 1 ? 1 : (np > Pmax ? Pmax : np);
        float tau = INFINITY;
        if (P < L) {
            uint32_t sP;
            if (P <= FEAT_K) {
                sP = __shfl_sync(0xffffffffu, fv, P - 1);
            } else if (P <= 48 && warp_small_kvals(load32, L, P, kv) >= 0) {
                sP = kv[P - 1];
                __syncwarp();
            } else {
                auto none = [](int, uint64_t) {};
                sP = (uint32_t)(warp_topk(load, L, P, none, hist, bb) >> 32);
            }
            tau = unordered_f32(sP) + (err ? 2.f * err[q] : 0.f);
        }
        const int n = collect_lists(ss, L, tau, ck, lane);
        if (n > RSW_CAND) {
            if (lane == 0) redo[1 + atomicAdd(&redo[0], 1)] = (int32_t)q;
        } else {
            exact_top_p(q, n, P, Pmax, ck, Q, Cc, d, spherical, probes, nullptr, lane);
        }
        __syncwarp();  // ss and ck are reused by the warp's next query
    }
}

// The predictor's distances (Sec. 4.2.1): per query the FEAT_K smallest list
// scores, ascending, from the given score matrix (the tensor-core scores,
// within their bound of the exact ones); for L2 the query's squared norm,
// which the ranking score leaves out, is added back.  One warp per query.
__global__ void __launch_bounds__(256) k_feat_scores(const float* __restrict__ scores, const float* __restrict__ Q,
                                                     int d, int spherical, int64_t nq, int L,
                                                     float* __restrict__ out) {
    __shared__ uint32_t hist[8][256];
    __shared__ uint64_t bb[8][32];
    __shared__ uint64_t kk[8][FEAT_K];
    __shared__ uint32_t kv[8][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * 8 + w;
    if (q >= nq) return;
    const float* row = scores + q * L;
    auto load = [&](int c) -> uint64_t { return ((uint64_t)ordered_f32(row[c]) << 32) | (uint32_t)c; };
    auto load32 = [&](int c) -> uint32_t { return ordered_f32(row[c]); };
    auto emit = [&](int i, uint64_t k) { kk[w][i] = k; };
    uint32_t v;  // this lane's distance (ordered image) in ascending order
    if (L > FEAT_K && warp_small_kvals(load32, L, FEAT_K, kv[w]) >= 0) {
        v = kv[w][lane];
    } else {
        if (L > FEAT_K) warp_topk(load, L, FEAT_K, emit, hist[w], bb[w]);
        else kk[w][lane] = load(lane);  // L == FEAT_K (the predictor needs 32 lists)
        __syncwarp();
        v = (uint32_t)(warp_sort_key(kk[w][lane], lane) >> 32);
    }
    float qq = 0.f;
    if (!spherical) {
        for (int t = lane; t < d; t += 32) qq = fmaf(Q[q * d + t], Q[q * d + t], qq);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qq += __shfl_xor_sync(0xffffffffu, qq, o);
    }
    out[q * FEAT_K + lane] = unordered_f32(v) + qq;
}

// ------------------------------------------------------------------ a2: quantised LUTs
// FP32 rule of the table entries, every op separately rounded:
//   L2: u_t = q_t - c_t, acc += (u_t - C_jit)^2 over t ascending
//   IP: u_t = q_t,       acc += u_t C_jit,                        T = -acc
// The row operand u (the dsub values of subspace j) is formed once per row;
// each entry is then the same sequence of rounded ops as written above.

struct LutArgs {
    const float* Q;
    int64_t nq;
    int d, M, dsub, ip, Pmax;
    const int32_t* probes;
    const int32_t* nprobe_q;
    int Pfix;
    const float* c_mean;
    const float* cb;
    int L;
    // optional compact work: pairs e = q * Pmax + r, two ranges (NULL: every
    // (q, r < P_q))
    const uint32_t* pairs0;
    const int64_t* npairs0;
    const uint32_t* pairs1;
    const int64_t* npairs1;
};

// Item i of the LUT pass: its (query, rank) flat index, or -1 if it does no work.
__device__ __forceinline__ int64_t lut_item(const LutArgs& A, int64_t i, int64_t n0) {
    if (A.pairs0) return i < n0 ? (int64_t)A.pairs0[i] : (int64_t)A.pairs1[i - n0];
    return i;
}

__device__ __forceinline__ int64_t lut_items(const LutArgs& A, int64_t* n0) {
    if (A.pairs0) {
        *n0 = *A.npairs0;
        return *n0 + *A.npairs1;
    }
    *n0 = 0;
    return A.nq * A.Pmax;
}

__device__ __forceinline__ int probes_of(const LutArgs& A, int64_t q) {
    int P = A.nprobe_q ? A.nprobe_q[q] : A.Pfix;
    return P < 1 ? 1 : (P > A.Pmax ? A.Pmax : P);
}

// Codebook row stride in shared memory.  dsub = 2: 34 floats (codewords
// 8-byte aligned; a half-warp reading 16 consecutive rows with 8-byte loads
// covers all 32 banks once); else 16 dsub + 1 (odd: 32 consecutive rows fall
// in distinct banks).
__host__ __device__ __forceinline__ int cb_ld(int dsub) { return dsub == 2 ? 34 : PQ_K * dsub + 1; }

__device__ __forceinline__ void stage_codebook(const LutArgs& A, float* cbs) {
    const int ld = cb_ld(A.dsub), rowlen = PQ_K * A.dsub;
    for (int e = threadIdx.x; e < A.M * rowlen; e += blockDim.x) {
        const int j = e / rowlen;
        cbs[j * ld + (e - j * rowlen)] = A.cb[e];
    }
    __syncthreads();
}

// The 16 FP32 entries of one subspace: qj, cj = the query's and the list
// centroid's values of the subspace, cw = its codebook row in shared memory.
// DS = dsub when fixed at compile time (2: 8-byte loads; qj and cj 8-byte
// aligned), 0 = read from dsub.
template <int DS>
__device__ __forceinline__ void row_table(int dsub, int ip, const float* __restrict__ qj,
                                          const float* __restrict__ cj, const float* cw, float (&T)[PQ_K]) {
    if constexpr (DS == 2) {
        const float2 qv = *reinterpret_cast<const float2*>(qj);
        float u0 = qv.x, u1 = qv.y;
        if (!ip) {
            const float2 cv = *reinterpret_cast<const float2*>(cj);
            u0 = __fsub_rn(u0, cv.x);
            u1 = __fsub_rn(u1, cv.y);
        }
#pragma unroll
        for (int i = 0; i < PQ_K; ++i) {
            const float2 c = *reinterpret_cast<const float2*>(cw + 2 * i);
            float acc = 0.f;
            if (ip) {
                acc = __fadd_rn(acc, __fmul_rn(u0, c.x));
                acc = __fadd_rn(acc, __fmul_rn(u1, c.y));
                T[i] = -acc;
            } else {
                // 0 + e0^2 is e0^2 exactly (a square is +0 or more), so the sum
                // from 0 needs one addition; both differences and both squares
                // as packed pairs
                const float2 e = f2_sub(make_float2(u0, u1), c);
                const float2 e2 = f2_mul(e, e);
                T[i] = __fadd_rn(e2.x, e2.y);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < PQ_K; ++i) T[i] = 0.f;
        for (int t = 0; t < dsub; ++t) {
            const float u = ip ? qj[t] : __fsub_rn(qj[t], cj[t]);
#pragma unroll
            for (int i = 0; i < PQ_K; ++i) {
                const float c = cw[i * dsub + t];
                if (ip) {
                    T[i] = __fadd_rn(T[i], __fmul_rn(u, c));
                } else {
                    const float e = __fsub_rn(u, c);
                    T[i] = __fadd_rn(T[i], __fmul_rn(e, e));
                }
            }
        }
        if (ip) {
#pragma unroll
            for (int i = 0; i < PQ_K; ++i) T[i] = -T[i];
        }
    }
}

// u8 entry min(255, floor((T - m) a + 1/2)) of four table entries, packed.
// T >= m, so the argument of floor is positive (or NaN, which converts to 0
// either way) and a conversion rounding down gives floor directly.
__device__ __forceinline__ uint32_t quant4(const float* T, float mn, float a) {
    uint32_t v[4];
#pragma unroll
    for (int i = 0; i < 4; i += 2) {  // (T - m) a + 1/2 of two entries as packed pairs
        const float2 x = f2_add(f2_mul(f2_sub(make_float2(T[i], T[i + 1]), make_float2(mn, mn)), make_float2(a, a)),
                                make_float2(0.5f, 0.5f));
        v[i] = min(__float2uint_rd(x.x), 255u);
        v[i + 1] = min(__float2uint_rd(x.y), 255u);
    }
    return __byte_perm(__byte_perm(v[0], v[1], 0x0040), __byte_perm(v[2], v[3], 0x0040), 0x5410);
}

// Integer bias floor(S a + 1/2) of one (query, list), S = sum_j m_j in
// ascending j (+ -<q, c_p> first for IP), clamped to +-2^30.
__device__ __forceinline__ int32_t lut_bias(const LutArgs& A, const float* __restrict__ qv, const float* __restrict__ cp,
                                            const float* mins, float a) {
    float S = 0.f;
    if (A.ip) {
        float dot = 0.f;
        for (int t = 0; t < A.d; ++t) dot = __fadd_rn(dot, __fmul_rn(qv[t], cp[t]));
        S = -dot;
    }
    for (int j = 0; j < A.M; ++j) S = __fadd_rn(S, mins[j]);
    float bf = floorf(__fadd_rn(__fmul_rn(S, a), 0.5f));
    bf = fminf(fmaxf(bf, -1073741824.f), 1073741823.f);
    return (int32_t)bf;
}

// Two-pass tables when a query's tables do not fit one CTA's shared memory
// (many probes): a warp per item (query, probe rank), lane l computing the
// rows j = l, l + 32, ... (M <= KSC_MAX_M), no block barrier.  Pass 1: the
// largest row range of each query, R_q (a warp maximum per item, then one
// global atomic maximum; R >= 0, so the bit order is the value order).
constexpr int LUT_WARPS = 8;

template <int DS>
__global__ void __launch_bounds__(LUT_WARPS * 32) k_lut_range(LutArgs A, uint32_t* __restrict__ range_bits) {
    extern __shared__ float cbs[];
    stage_codebook(A, cbs);
    const int ld = cb_ld(A.dsub);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t n0;
    const int64_t items = lut_items(A, &n0);
    for (int64_t i = (int64_t)blockIdx.x * LUT_WARPS + warp; i < items; i += (int64_t)gridDim.x * LUT_WARPS) {
        const int64_t item = lut_item(A, i, n0);
        const int64_t q = item / A.Pmax;
        const int r = (int)(item - q * A.Pmax);
        const int p = A.probes[item];
        if (r >= probes_of(A, q) || p < 0 || p >= A.L) continue;  // invalid probe ids are skipped (warp-uniform)
        float R = 0.f;
        for (int j = lane; j < A.M; j += 32) {
            float T[PQ_K];
            row_table<DS>(A.dsub, A.ip, A.Q + q * A.d + j * A.dsub, A.c_mean + (int64_t)p * A.d + j * A.dsub,
                          cbs + j * ld, T);
            float mn = T[0], mx = T[0];
#pragma unroll
            for (int e = 1; e < PQ_K; ++e) { mn = fminf(mn, T[e]); mx = fmaxf(mx, T[e]); }
            R = fmaxf(R, __fsub_rn(mx, mn));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) R = fmaxf(R, __shfl_xor_sync(0xffffffffu, R, o));
        if (lane == 0 && R > 0.f) atomicMax(&range_bits[q], __float_as_uint(R));
    }
}

// Pass 2: u8 tables Q = min(255, floor((T - m_j) a + 1/2)), a = 255 / R_q,
// then the item's bias from its row minima (summed in ascending j by lane 0,
// the FP32 rule's order).
template <int DS>
__global__ void __launch_bounds__(LUT_WARPS * 32) k_lut_quant(LutArgs A, const uint32_t* __restrict__ range_bits,
                                                              uint8_t* __restrict__ lut, int32_t* __restrict__ bias,
                                                              float* __restrict__ scale) {
    extern __shared__ float cbs[];
    __shared__ float s_min[LUT_WARPS][KSC_MAX_M];
    stage_codebook(A, cbs);
    const int ld = cb_ld(A.dsub);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t n0;
    const int64_t items = lut_items(A, &n0);
    for (int64_t i = (int64_t)blockIdx.x * LUT_WARPS + warp; i < items; i += (int64_t)gridDim.x * LUT_WARPS) {
        const int64_t item = lut_item(A, i, n0);
        const int64_t q = item / A.Pmax;
        const int r = (int)(item - q * A.Pmax);
        const int p = A.probes[item];
        if (r >= probes_of(A, q) || p < 0 || p >= A.L) continue;  // warp-uniform
        const float Rq = __uint_as_float(range_bits[q]);
        const float a = (Rq == 0.f) ? 1.f : __fdiv_rn(255.f, Rq);
        for (int j = lane; j < A.M; j += 32) {
            float T[PQ_K];
            row_table<DS>(A.dsub, A.ip, A.Q + q * A.d + j * A.dsub, A.c_mean + (int64_t)p * A.d + j * A.dsub,
                          cbs + j * ld, T);
            float mn = T[0];
#pragma unroll
            for (int e = 1; e < PQ_K; ++e) mn = fminf(mn, T[e]);
            reinterpret_cast<uint4*>(lut + item * (int64_t)A.M * PQ_K)[j] =
                make_uint4(quant4(T, mn, a), quant4(T + 4, mn, a), quant4(T + 8, mn, a), quant4(T + 12, mn, a));
            s_min[warp][j] = mn;
        }
        __syncwarp();
        if (lane == 0) {
            bias[item] = lut_bias(A, A.Q + q * A.d, A.c_mean + (int64_t)p * A.d, s_min[warp], a);
            if (r == 0) scale[q] = a;
        }
        __syncwarp();  // s_min is read before the warp's next item overwrites it
    }
}

// Persistent CTAs, one query at a time, when all of a query's tables fit in
// shared memory: the codebook is staged once per CTA; the FP32 tables of the
// query's P_q probes are computed once, their largest range gives the scale,
// and they are quantised from shared memory (same FP32 rule, same results as
// the two-pass kernels above).  Rows of 16 entries sit 20 floats apart (16-byte
// aligned; 8 consecutive rows of a 128-bit access fall in distinct banks).  A
// thread walks rows (r, j) = (probe rank, subspace) by a fixed step, no
// division.  Two barriers per query: the next query's vector is loaded into
// the other of two buffers while this one is quantised.
constexpr int LUT_TROW = 20;

template <int DS>
__global__ void __launch_bounds__(256) k_lut_fused(LutArgs A, int Pb, int Pm, uint8_t* __restrict__ lut,
                                                   int32_t* __restrict__ bias, float* __restrict__ scale) {
    extern __shared__ __align__(16) float fsm[];
    const int M = A.M;
    const int ld = cb_ld(A.dsub);
    const int dpad = (A.d + 3) & ~3;
    float* cbs = fsm;                                                  // M x ld
    float* T = cbs + (((size_t)M * ld + 3) & ~(size_t)3);              // Pb x M rows, LUT_TROW apart
    float* mins = T + (size_t)Pb * M * LUT_TROW;                       // Pm x M
    float* qsb = mins + (((size_t)Pm * M + 3) & ~(size_t)3);           // 2 x dpad
    int32_t* prb = reinterpret_cast<int32_t*>(qsb + 2 * dpad);         // 2 x Pm probe ids
    __shared__ uint32_t s_rbits[2];
    const int r0 = threadIdx.x / M, j0 = threadIdx.x - r0 * M;         // first row of this thread
    const int dr = blockDim.x / M, dj = blockDim.x - dr * M;           // step of blockDim.x rows
    int64_t q = blockIdx.x;
    if (q < A.nq) {
        for (int t = threadIdx.x; t < A.d; t += blockDim.x) qsb[t] = A.Q[q * A.d + t];
        for (int r = threadIdx.x; r < Pm; r += blockDim.x) prb[r] = A.probes[q * A.Pmax + r];
    }
    if (threadIdx.x == 0) s_rbits[0] = 0u;
    stage_codebook(A, cbs);  // ends with __syncthreads
    for (int buf = 0; q < A.nq; q += gridDim.x, buf ^= 1) {
        const float* qs = qsb + buf * dpad;
        // the tables of the first Pb probes are kept for the quantisation
        // pass; those of later probes (a query with more) are computed again
        const int P = min(probes_of(A, q), Pm);
        const int nstored = Pb * M;
        const int32_t* pr = prb + buf * Pm;  // the query's probes, staged in shared memory
        float R = 0.f;
        {
            int r = r0, j = j0;
            for (int row = threadIdx.x; row < P * M; row += blockDim.x) {
                const int p = pr[r];
                float* Tr = T + (size_t)row * LUT_TROW;
                const bool stored = row < nstored;
                if (p < 0 || p >= A.L) {
                    if (stored)
#pragma unroll
                        for (int i = 0; i < PQ_K; i += 4) *reinterpret_cast<float4*>(Tr + i) = make_float4(0.f, 0.f, 0.f, 0.f);
                    mins[row] = 0.f;
                } else {
                    float Tv[PQ_K];
                    row_table<DS>(A.dsub, A.ip, qs + j * A.dsub, A.c_mean + (int64_t)p * A.d + j * A.dsub,
                                  cbs + j * ld, Tv);
                    float mn = Tv[0], mx = Tv[0];
#pragma unroll
                    for (int i = 1; i < PQ_K; ++i) {
                        mn = fminf(mn, Tv[i]);
                        mx = fmaxf(mx, Tv[i]);
                    }
                    if (stored)
#pragma unroll
                        for (int i = 0; i < PQ_K; i += 4)
                            *reinterpret_cast<float4*>(Tr + i) = make_float4(Tv[i], Tv[i + 1], Tv[i + 2], Tv[i + 3]);
                    mins[row] = mn;
                    R = fmaxf(R, __fsub_rn(mx, mn));
                }
                j += dj;
                r += dr;
                if (j >= M) {
                    j -= M;
                    ++r;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) R = fmaxf(R, __shfl_xor_sync(0xffffffffu, R, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&s_rbits[buf], __float_as_uint(R));
        __syncthreads();
        const float Rq = __uint_as_float(s_rbits[buf]);
        const float a = (Rq == 0.f) ? 1.f : __fdiv_rn(255.f, Rq);
        // the next query's vector into the other buffer (its last readers
        // passed the barrier above)
        const int64_t qn = q + gridDim.x;
        float* qs_next = qsb + (buf ^ 1) * dpad;
        const bool pre = qn < A.nq && threadIdx.x < A.d;
        const float nx = pre ? A.Q[qn * A.d + threadIdx.x] : 0.f;
        if (threadIdx.x == 0) s_rbits[buf ^ 1] = 0u;
        {
            int r = r0, j = j0;
            for (int row = threadIdx.x; row < P * M; row += blockDim.x) {
                const float mn = mins[row];
                float Tv[PQ_K];
                bool ok = true;
                if (row < nstored) {
                    const float* Tr = T + (size_t)row * LUT_TROW;
#pragma unroll
                    for (int i = 0; i < PQ_K; i += 4) {
                        const float4 v = *reinterpret_cast<const float4*>(Tr + i);
                        Tv[i] = v.x;
                        Tv[i + 1] = v.y;
                        Tv[i + 2] = v.z;
                        Tv[i + 3] = v.w;
                    }
                } else {
                    const int p = pr[r];
                    ok = p >= 0 && p < A.L;
                    if (ok)
                        row_table<DS>(A.dsub, A.ip, qs + j * A.dsub, A.c_mean + (int64_t)p * A.d + j * A.dsub,
                                      cbs + j * ld, Tv);
                }
                if (ok)
                    reinterpret_cast<uint4*>(lut + (q * A.Pmax + r) * (int64_t)M * PQ_K)[j] = make_uint4(
                        quant4(Tv, mn, a), quant4(Tv + 4, mn, a), quant4(Tv + 8, mn, a), quant4(Tv + 12, mn, a));
                j += dj;
                r += dr;
                if (j >= M) {
                    j -= M;
                    ++r;
                }
            }
        }
        // biases by the last threads (those with the fewest rows above)
        for (int r = blockDim.x - 1 - threadIdx.x; r < P; r += blockDim.x) {
            const int p = pr[r];
            if (p < 0 || p >= A.L) continue;
            bias[q * A.Pmax + r] = lut_bias(A, qs, A.c_mean + (int64_t)p * A.d, mins + r * M, a);
        }
        if (threadIdx.x == 0) scale[q] = a;
        if (pre) qs_next[threadIdx.x] = nx;
        if (qn < A.nq) {
            for (int t = threadIdx.x + blockDim.x; t < A.d; t += blockDim.x) qs_next[t] = A.Q[qn * A.d + t];
            for (int r = threadIdx.x; r < Pm; r += blockDim.x) prb[(buf ^ 1) * Pm + r] = A.probes[qn * A.Pmax + r];
        }
        __syncthreads();  // the next query reuses the shared tables
    }
}

static size_t lut_fused_smem(int M, int dsub, int d, int Pb, int Pm) {
    return sizeof(float) * ((((size_t)M * cb_ld(dsub) + 3) & ~(size_t)3) + (size_t)Pb * M * LUT_TROW +
                            (((size_t)Pm * M + 3) & ~(size_t)3) + 2 * (((size_t)d + 3) & ~(size_t)3)) +
           sizeof(int32_t) * 2 * (size_t)Pm;
}

// 8-byte row loads need dsub = 2 and an 8-byte aligned query matrix.
static bool lut_ds2(const LutArgs& A) { return A.dsub == 2 && (reinterpret_cast<uintptr_t>(A.Q) & 7) == 0; }

static int launch_luts(const LutArgs& A, uint32_t* rb, uint8_t* lut, int32_t* bias, float* scale, cudaStream_t st);

// ------------------------------------------------------------------ code access
__device__ __forceinline__ int nibble_of(const uint8_t* __restrict__ blk, int M, int j, int v) {
    uint8_t byte = blk[j * 16 + (v >> 1)];
    return (v & 1) ? (byte >> 4) : (byte & 15);
}

__device__ __forceinline__ int32_t scalar_dist(const uint8_t* __restrict__ lutp, int32_t b,
                                               const uint8_t* __restrict__ blk, int M, int v) {
    int32_t D = b;
    for (int j = 0; j < M; ++j) D += lutp[j * 16 + nibble_of(blk, M, j, v)];
    return D;
}

// ------------------------------------------------------------------ candidate-key selection
// The need smallest keys of distance word h among keys[0..N) (the others
// mapped above every key, uniquely by index), into out[0..need) unless out
// is null; returns the need-th.  The tie case of warp_topk_hi.
__device__ __forceinline__ uint64_t warp_topk_tied(const uint64_t* __restrict__ keys, int N, int need, uint32_t h,
                                                uint64_t* out, uint32_t* hist, uint64_t* bb) {
    auto load_t = [&](int i) -> uint64_t {
        const uint64_t k = keys[i];
        return (uint32_t)(k >> 32) == h ? k : ((0xffffffffull << 32) | (uint32_t)i);
    };
    auto emit_t = [&](int i, uint64_t k) {
        if (out) out[i] = k;
    };
    return warp_topk(load_t, N, need, emit_t, hist, bb);
}

// The K smallest (0 < K < N) of N unique candidate keys keys[0..N) (high word:
// the integer distance + 2^31, below 2^32 - 1; low word: the vector id), by
// one warp, as warp_topk but with the range, histogram and emission decided
// on the keys' high words alone (32-bit loads and compares: the distance
// range always spans more than the id bits matter for) until the K-th key's
// bin holds at most 32 keys, which are sorted on their full 64 bits.  A bin
// narrowed to a single distance with more than 32 keys in it (ties) hands the
// rest to warp_topk over those keys.  Writes the K smallest to dst[0..K) in
// no particular order (nothing if dst is null) and returns the K-th.
__device__ uint64_t warp_topk_hi(const uint64_t* __restrict__ keys, int N, int K, uint64_t* dst, uint32_t* hist,
                                 uint64_t* bb) {
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t* hw = reinterpret_cast<const uint32_t*>(keys) + 1;  // key i's high word at hw[2 i]
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int i0 = 0; i0 < N; i0 += 32 * TOPK_U) {
        uint32_t h[TOPK_U];
#pragma unroll
        for (int u = 0; u < TOPK_U; ++u) {
            const int i = i0 + 32 * u + lane;
            h[u] = i < N ? hw[2 * i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < TOPK_U; ++u)
            if (i0 + 32 * u + lane < N) {
                lo = min(lo, h[u]);
                hi = max(hi, h[u]);
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    int out = 0, need = K;
    while (lo < hi) {
        int shift = 0;
        while (((hi - lo) >> shift) >= 256u) ++shift;
        for (int b = lane; b < 256; b += 32) hist[b] = 0u;
        __syncwarp();
        for (int i0 = 0; i0 < N; i0 += 32 * TOPK_U) {
            uint32_t h[TOPK_U];
#pragma unroll
            for (int u = 0; u < TOPK_U; ++u) {
                const int i = i0 + 32 * u + lane;
                h[u] = i < N ? hw[2 * i] : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < TOPK_U; ++u)
                if (i0 + 32 * u + lane < N && h[u] >= lo && h[u] <= hi) atomicAdd(&hist[(h[u] - lo) >> shift], 1u);
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
        const uint32_t blo = lo + ((uint32_t)B << shift);
        const uint32_t bhi = (hi - blo < (1u << shift)) ? hi : blo + ((1u << shift) - 1u);
        const bool last = inB <= 32;
        int nb = 0;
        for (int i0 = 0; i0 < N; i0 += 32 * TOPK_U) {
            uint32_t h[TOPK_U];
#pragma unroll
            for (int u = 0; u < TOPK_U; ++u) {
                const int i = i0 + 32 * u + lane;
                h[u] = i < N ? hw[2 * i] : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < TOPK_U; ++u) {
                const int i = i0 + 32 * u + lane;
                const bool e = i < N && h[u] >= lo && h[u] < blo;
                const bool g = last && i < N && h[u] >= blo && h[u] <= bhi;
                const uint32_t me = __ballot_sync(0xffffffffu, e), mg = __ballot_sync(0xffffffffu, g);
                if (e && dst) dst[out + __popc(me & below)] = keys[i];
                if (g) bb[nb + __popc(mg & below)] = keys[i];
                out += __popc(me);
                nb += __popc(mg);
            }
        }
        need -= lt;
        if (last) {
            __syncwarp();
            const uint64_t v = warp_sort_key(lane < inB ? bb[lane] : KEY_NONE, lane);
            if (lane < need && dst) dst[out + lane] = v;
            const uint64_t kth = __shfl_sync(0xffffffffu, v, need - 1);
            __syncwarp();
            return kth;
        }
        lo = blo;
        hi = bhi;
        __syncwarp();
    }
    // one distance left with more keys than the sort takes: the need smallest
    // of its keys by their ids
    return warp_topk_tied(keys, N, need, lo, dst ? dst + out : nullptr, hist, bb);
}

// ------------------------------------------------------------------ threshold
// Per query, after the scan of its nearest list(s) with no filter: the R-th
// smallest of the keys found so far bounds the R-th smallest key of the whole
// search from above (any subset with at least R members gives such a bound);
// the scan of the remaining lists keeps only keys at or below it.  Fewer than
// R keys: no bound (all ones).  One warp per query.  Nothing above the R-th
// key can enter the final R, so the store keeps only the R keys at or below it
// (gathered in `scratch`, a row of Rmax keys per query, then copied back),
// unless it overflowed (the final select then redoes the query).
constexpr int SW_WARPS = 8;        // queries per CTA of the warp selection kernels
constexpr int SW_MAX_KEYS = 2048;  // expected keys per query up to which a warp selects

__global__ void __launch_bounds__(SW_WARPS * 32) k_threshold(ScanArgs A, int Rmax, int32_t* __restrict__ cnt,
                                                             uint64_t* __restrict__ cand, int cap,
                                                             uint64_t* __restrict__ scratch,
                                                             uint64_t* __restrict__ thr) {
    __shared__ uint32_t hist[SW_WARPS][256];
    __shared__ uint64_t bb[SW_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * SW_WARPS + w;
    if (q >= A.nq) return;
    const int R = rerank_of(A.rerank_q, A.Rfix, A.Rmin, Rmax, q);
    const int n0 = cnt[q];
    const int n = min(n0, cap);  // an overflowed store still bounds the R-th key
    const bool ovf = n0 > cap;
    uint64_t* cq = cand + q * cap;
    uint64_t t = KEY_NONE;
    if (n == R) {
        uint64_t m = 0ull;
        for (int i = lane; i < n; i += 32) m = cq[i] > m ? cq[i] : m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t y = __shfl_xor_sync(0xffffffffu, m, o);
            m = y > m ? y : m;
        }
        t = m;
    } else if (n > R) {
        uint64_t* sq = scratch + q * Rmax;
        t = warp_topk_hi(cq, n, R, ovf ? nullptr : sq, hist[w], bb[w]);
        if (!ovf) {
            __syncwarp();
            for (int i = lane; i < R; i += 32) cq[i] = sq[i];
            if (lane == 0) cnt[q] = R;
        }
    }
    if (lane == 0) thr[q] = t;
}

// The same with one CTA per query, for queries with many keys (NT threads:
// 1024 when the batch is too small to fill the GPU with 256-thread CTAs).
template <int NT>
__global__ void __launch_bounds__(NT) k_threshold_cta(ScanArgs A, int Rmax, int32_t* __restrict__ cnt,
                                                       uint64_t* __restrict__ cand, int cap,
                                                       uint64_t* __restrict__ scratch,
                                                       uint64_t* __restrict__ thr) {
    __shared__ uint32_t hist[256];
    __shared__ uint64_t bb[32];
    __shared__ unsigned long long s_m;
    const int64_t q = blockIdx.x;
    const int R = rerank_of(A.rerank_q, A.Rfix, A.Rmin, Rmax, q);
    const int n0 = cnt[q];
    const int n = min(n0, cap);
    const bool ovf = n0 > cap;
    uint64_t* cq = cand + q * cap;
    uint64_t t = KEY_NONE;
    if (n == R) {
        if (threadIdx.x == 0) s_m = 0ull;
        __syncthreads();
        unsigned long long m = 0ull;
        for (int i = threadIdx.x; i < n; i += blockDim.x) m = cq[i] > m ? cq[i] : m;
        atomicMax(&s_m, m);
        __syncthreads();
        t = s_m;
    } else if (n > R) {
        uint64_t* sq = scratch + q * Rmax;
        auto load = [&](int i) -> uint64_t { return cq[i]; };
        auto emit = [&](int i, uint64_t k) {
            if (!ovf) sq[i] = k;
        };
        t = block_topk(load, n, R, emit, hist, bb);
        if (!ovf) {
            for (int i = threadIdx.x; i < R; i += blockDim.x) cq[i] = sq[i];
            if (threadIdx.x == 0) cnt[q] = R;
        }
    }
    if (threadIdx.x == 0) thr[q] = t;
}

// ------------------------------------------------------------------ work list (cluster-major)
// pairs of (query, probe rank) grouped by list; items = (list, query group,
// block tile).
// Work lists of both parts of every query's probe ranks, in one pass: a warp
// per query finds the end of the unfiltered first part and counts the pairs
// of each part per list.  First part (plain search): the fewest nearest lists
// holding S = max(NEAR_KEYS_PER_R * R, N / NEAR_SHARE_DIV) keys, N = the keys
// the query probes.  The R-th key of a first set of S keys sits near the R/S
// quantile of the nearest keys and the remaining lists are farther, so at most
// about N R / S of their keys pass it: a few R.  S is at most half the
// candidate store, and the first part never holds more keys than the store
// (at least one list).  Hybrid search: the first `rs` ranks.  split[q] (plain
// only) records the boundary for k_fill_parts.

__global__ void k_count_parts(ScanArgs A, int Rmax, int cap, int rs, int32_t* __restrict__ split,
                              int32_t* __restrict__ cntA, int32_t* __restrict__ cntB,
                              int32_t* __restrict__ near_cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= A.nq) return;
    const int P = nprobe_of(A, q);
    const int32_t* pr = A.probes + q * A.Pmax;
    int b = rs;
    if (split) {
        long long total = 0;
        for (int r = lane; r < P; r += 32) total += list_size(A, pr[r]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        long long target = (long long)NEAR_KEYS_PER_R * rerank_of(A.rerank_q, A.Rfix, A.Rmin, Rmax, q);
        target = max(target, total / NEAR_SHARE_DIV);
        target = min(target, (long long)cap / 2);
        // first rank r whose keys-before reach the target, or (r > 0) whose list
        // would overflow the store
        long long acc = 0;
        int bnd = P;
        for (int r0 = 0; r0 < P; r0 += 32) {
            const int r = r0 + lane;
            const long long n = r < P ? list_size(A, pr[r]) : 0;
            long long incl = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const long long before = acc + incl - n;
            const bool stop = r < P && (before >= target || (r > 0 && before + n > cap));
            const uint32_t m = __ballot_sync(0xffffffffu, stop);
            if (m) {
                bnd = r0 + __ffs(m) - 1;
                break;
            }
            acc += __shfl_sync(0xffffffffu, incl, 31);
        }
        b = bnd < 1 ? 1 : bnd;
        if (lane == 0) split[q] = b;
    }
    long long nn = 0;
    for (int r = lane; r < P; r += 32) {
        const int p = pr[r];
        if (p >= 0 && p < A.L) atomicAdd(r < b ? &cntA[p] : &cntB[p], 1);
        if (r < b) nn += list_size(A, p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    // the unfiltered scan writes every key of the first part at a fixed place
    if (lane == 0) near_cnt[q] = (int32_t)(nn < 0x7fffffffll ? nn : 0x7fffffffll);
}


// exclusive scans: pair_off = scan(cnt); item_off = scan(ceil(cnt/QG) * ntiles)
// Several work lists at once: CTA i scans cnt + i L into pair_off / item_off +
// i (L + 1) and clears fill + i L; the first list's items hold QG0 queries and
// tiles of TB0 blocks, the others' QG1 and TB1.
__global__ void __launch_bounds__(1024) k_scan_lists(const int32_t* __restrict__ cnt0, const int32_t* __restrict__ list_n,
                                                     int L, int QG0, int QG1, int TB0, int TB1,
                                                     int64_t* __restrict__ pair_off0, int64_t* __restrict__ item_off0,
                                                     int32_t* __restrict__ fill0) {
    const int TB = blockIdx.x == 0 ? TB0 : TB1;  // tile length of this CTA's work list
    const int QG = blockIdx.x == 0 ? QG0 : QG1;  // queries per item
    const int32_t* cnt = cnt0 + (size_t)blockIdx.x * L;
    int64_t* pair_off = pair_off0 + (size_t)blockIdx.x * (L + 1);
    int64_t* item_off = item_off0 + (size_t)blockIdx.x * (L + 1);
    int32_t* fill = fill0 + (size_t)blockIdx.x * L;
    __shared__ int64_t s_p[1024], s_i[1024];
    const int per = (L + 1023) / 1024;
    const int c0 = threadIdx.x * per;
    int64_t sp = 0, si = 0;
    for (int c = c0; c < c0 + per && c < L; ++c) {
        sp += cnt[c];
        int nb = (list_n[c] + 31) >> 5;
        int nt = (nb + TB - 1) / TB;
        si += (int64_t)((cnt[c] + QG - 1) / QG) * nt;
    }
    s_p[threadIdx.x] = sp;
    s_i[threadIdx.x] = si;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t vp = threadIdx.x >= o ? s_p[threadIdx.x - o] : 0;
        int64_t vi = threadIdx.x >= o ? s_i[threadIdx.x - o] : 0;
        __syncthreads();
        s_p[threadIdx.x] += vp;
        s_i[threadIdx.x] += vi;
        __syncthreads();
    }
    int64_t bp = s_p[threadIdx.x] - sp, bi = s_i[threadIdx.x] - si;
    for (int c = c0; c < c0 + per && c < L; ++c) {
        pair_off[c] = bp;
        item_off[c] = bi;
        fill[c] = 0;
        bp += cnt[c];
        int nb = (list_n[c] + 31) >> 5;
        int nt = (nb + TB - 1) / TB;
        bi += (int64_t)((cnt[c] + QG - 1) / QG) * nt;
    }
    if (threadIdx.x == 1023) {
        pair_off[L] = s_p[1023];
        item_off[L] = s_i[1023];
    }
}

__global__ void k_fill_parts(ScanArgs A, int rs, const int32_t* __restrict__ split,
                             const int64_t* __restrict__ offA, int32_t* __restrict__ fillA, uint32_t* __restrict__ pairsA,
                             const int64_t* __restrict__ offB, int32_t* __restrict__ fillB,
                             uint32_t* __restrict__ pairsB) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= A.nq * A.Pmax) return;
    int64_t q = e / A.Pmax;
    int r = (int)(e - q * A.Pmax);
    if (r >= nprobe_of(A, q)) return;
    const int p = A.probes[e];
    if (p < 0 || p >= A.L) return;
    const bool first = r < (split ? split[q] : rs);
    const int slot = atomicAdd(first ? &fillA[p] : &fillB[p], 1);
    (first ? pairsA : pairsB)[(first ? offA : offB)[p] + slot] = (uint32_t)e;  // e = q * Pmax + r
}

// ------------------------------------------------------------------ a3: LUT16 scan

// Eight lookups of one 16-entry u8 table t (4 registers, entry e in byte e)
// for the eight 4-bit codes of w (code of vector n in bits 4n..4n+3):
// lo = bytes T[c0..c3], hi = bytes T[c4..c7].  Two byte permutes fetch
// T[c & 7] and T[8 + (c & 7)], a third picks per byte by bit 3 of c.  A byte
// permute reads only the low 16 bits of its selector, so both halves come
// from one masked word and a shift.
__device__ __forceinline__ void lut16x8(uint32_t w, const uint4& t, uint32_t& lo, uint32_t& hi) {
    const uint32_t s0 = w & 0x77777777u;                            // entry index within a half
    const uint32_t s1 = s0 >> 16;
    const uint32_t k0 = ((w >> 1) & 0x44444444u) | 0x32103210u;     // byte n of a (n) or of b (4 + n)
    const uint32_t k1 = k0 >> 16;
    lo = prmt(prmt(t.x, t.y, s0), prmt(t.z, t.w, s0), k0);
    hi = prmt(prmt(t.x, t.y, s1), prmt(t.z, t.w, s1), k1);
}

// Add the 16 lookups of one (subspace, 16-byte code chunk) into the u16x2
// lane sums acc[m] = (vector 2m, vector 2m+1).
__device__ __forceinline__ void accum_chunk(const uint4& c, const uint4& t, uint32_t (&acc)[16]) {
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t lo, hi;
        lut16x8(w[k], t, lo, hi);
        acc[4 * k + 0] += prmt(lo, 0u, 0x4140u);
        acc[4 * k + 1] += prmt(lo, 0u, 0x4342u);
        acc[4 * k + 2] += prmt(hi, 0u, 0x4140u);
        acc[4 * k + 3] += prmt(hi, 0u, 0x4342u);
    }
}

// Two subspaces at once: each lane sum takes both widened lookups in one
// three-input add.
__device__ __forceinline__ void accum_pair(const uint4& c0, const uint4& t0, const uint4& c1, const uint4& t1,
                                           uint32_t (&acc)[16]) {
    const uint32_t w0[4] = {c0.x, c0.y, c0.z, c0.w};
    const uint32_t w1[4] = {c1.x, c1.y, c1.z, c1.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t lo0, hi0, lo1, hi1;
        lut16x8(w0[k], t0, lo0, hi0);
        lut16x8(w1[k], t1, lo1, hi1);
        acc[4 * k + 0] += prmt(lo0, 0u, 0x4140u) + prmt(lo1, 0u, 0x4140u);
        acc[4 * k + 1] += prmt(lo0, 0u, 0x4342u) + prmt(lo1, 0u, 0x4342u);
        acc[4 * k + 2] += prmt(hi0, 0u, 0x4140u) + prmt(hi1, 0u, 0x4140u);
        acc[4 * k + 3] += prmt(hi0, 0u, 0x4342u) + prmt(hi1, 0u, 0x4342u);
    }
}

// Reduce-scatter of the 16 u16x2 sums over the G lanes of a group: after it,
// group lane g holds the full sums of vectors V*g .. V*g+V-1 (V = 32/G) in
// out[0..V) (u16 values).
// The same lookups with the widening done by byte dot products (dp4a with a
// one-hot byte selector adds byte b of the looked-up word to a 32-bit sum):
// acc[v] is the sum of vector v.  The dot products issue on the FMA pipe, so
// the integer pipe keeps only the selector and permute work.
__device__ __forceinline__ void widen_add4(uint32_t x, uint32_t* acc) {
    acc[0] = __dp4a(x, 0x00000001u, acc[0]);
    acc[1] = __dp4a(x, 0x00000100u, acc[1]);
    acc[2] = __dp4a(x, 0x00010000u, acc[2]);
    acc[3] = __dp4a(x, 0x01000000u, acc[3]);
}

__device__ __forceinline__ void accum_chunk32(const uint4& c, const uint4& t, uint32_t (&acc)[32]) {
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t lo, hi;
        lut16x8(w[k], t, lo, hi);
        widen_add4(lo, acc + 8 * k);
        widen_add4(hi, acc + 8 * k + 4);
    }
}

__device__ __forceinline__ void accum_pair32(const uint4& c0, const uint4& t0, const uint4& c1, const uint4& t1,
                                             uint32_t (&acc)[32]) {
    accum_chunk32(c0, t0, acc);
    accum_chunk32(c1, t1, acc);
}

// Selectors of one code word w (eight 4-bit codes, vector n in bits 4n..4n+3)
// for lut16x8, computed once per word and shared by every query slot of a
// warp: (s0, s1, k0, k1).
__device__ __forceinline__ uint4 lut16_selectors(uint32_t w) {
    const uint32_t s0 = w & 0x77777777u;
    const uint32_t k0 = ((w >> 1) & 0x44444444u) | 0x32103210u;
    return make_uint4(s0, s0 >> 16, k0, k0 >> 16);
}

// The lookups of one word from its selectors: lo = T[c0..c3], hi = T[c4..c7].
__device__ __forceinline__ void lut16x8_sel(const uint4& s, const uint4& t, uint32_t& lo, uint32_t& hi) {
    lo = prmt(prmt(t.x, t.y, s.x), prmt(t.z, t.w, s.x), s.z);
    hi = prmt(prmt(t.x, t.y, s.y), prmt(t.z, t.w, s.y), s.w);
}

// Two subspaces j0, j1 from shared selectors (sel[k M + j]: word k of
// subspace j): the looked-up bytes of the same vector from both subspaces
// are interleaved by one byte permute, so one byte dot product adds two
// lookups to the vector's 32-bit sum (acc[v], v the vector of the block).
__device__ __forceinline__ void accum_pair_sel(const uint4* __restrict__ sel, int M, int j0, int j1, const uint4& t0,
                                               const uint4& t1, uint32_t (&acc)[32]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t lo0, hi0, lo1, hi1;
        lut16x8_sel(sel[k * M + j0], t0, lo0, hi0);
        lut16x8_sel(sel[k * M + j1], t1, lo1, hi1);
        uint32_t* a = acc + 8 * k;
        uint32_t x = prmt(lo0, lo1, 0x5140u), y = prmt(lo0, lo1, 0x7362u);
        a[0] = __dp4a(x, 0x00000101u, a[0]);
        a[1] = __dp4a(x, 0x01010000u, a[1]);
        a[2] = __dp4a(y, 0x00000101u, a[2]);
        a[3] = __dp4a(y, 0x01010000u, a[3]);
        x = prmt(hi0, hi1, 0x5140u);
        y = prmt(hi0, hi1, 0x7362u);
        a[4] = __dp4a(x, 0x00000101u, a[4]);
        a[5] = __dp4a(x, 0x01010000u, a[5]);
        a[6] = __dp4a(y, 0x00000101u, a[6]);
        a[7] = __dp4a(y, 0x01010000u, a[7]);
    }
}

__device__ __forceinline__ void accum_chunk_sel(const uint4* __restrict__ sel, int M, int j, const uint4& t,
                                                uint32_t (&acc)[32]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t lo, hi;
        lut16x8_sel(sel[k * M + j], t, lo, hi);
        widen_add4(lo, acc + 8 * k);
        widen_add4(hi, acc + 8 * k + 4);
    }
}

template <int G>
__device__ __forceinline__ void reduce_scatter(uint32_t (&acc)[16], int lane, uint32_t (&out)[32 / G]) {
    constexpr int V = 32 / G;
    int nreg = 16;
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) {
        if (nreg == 1) break;
        const int h = nreg >> 1;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < h) {
                uint32_t send = up ? acc[i] : acc[i + h];
                uint32_t keep = up ? acc[i + h] : acc[i];
                acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        nreg = h;
    }
    if constexpr (V == 1) {
        // G = 32: one register of two vectors left; split it over lane bit 0
        const bool odd = lane & 1;
        uint32_t send = odd ? (acc[0] & 0xffffu) : (acc[0] >> 16);
        uint32_t keep = odd ? (acc[0] >> 16) : (acc[0] & 0xffffu);
        out[0] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
    } else {
#pragma unroll
        for (int i = 0; i < V / 2; ++i) {
            out[2 * i] = acc[i] & 0xffffu;
            out[2 * i + 1] = acc[i] >> 16;
        }
    }
}


// Persistent, cluster-major scan with shared-memory staging of the codes.
// A warp takes one item = (list p, group of QG = 32/G queries that probe p,
// tile of at most TB blocks of p) and walks the tile in chunks of
// SCAN_CHUNK blocks.  Lane 0 bulk-copies each chunk's codes (contiguous in
// global memory) into the warp's own shared-memory buffer with cp.async.bulk,
// completing the warp's mbarrier; two buffers alternate so that the next
// chunk -- of this item or of the warp's next item -- is in flight while the
// current one is scanned.  Group lane g of query slot s holds the sub-LUTs of
// subspaces j = g + G*u (u < SMAX) in registers.  A key is formed only for a
// vector whose distance reaches its query's threshold, so ids are read from
// global memory only for those.  With no threshold (the first part of every
// query, O.thr null) every key is kept and written straight to its fixed place
// in the store (near_offset of its probe rank + its index in the list; the
// count is preset by k_count_parts), its id loaded before the block's lookups.
// No CTA-wide barrier: warps run independently.
constexpr int SCAN_WARPS = 8;
constexpr int SCAN_CHUNK_BYTES = 4096;           // per buffer, per warp
constexpr int SCAN_CHUNK_BYTES_SEL = 3072;       // the same with shared selectors (room for their buffer)
constexpr int SCAN_BUF_KEYS = 64;                // kept keys buffered per (warp, query slot)

// With 8 lanes per query the four query slots of a warp read the same code
// words: their selectors are computed once per block into a shared buffer of
// M x 64 bytes per warp.
template <int G>
__host__ __device__ constexpr bool scan_shared_sel() { return G == 8; }
template <int G>
__host__ __device__ constexpr int scan_chunk_bytes() { return scan_shared_sel<G>() ? SCAN_CHUNK_BYTES_SEL : SCAN_CHUNK_BYTES; }
constexpr uint32_t SCAN_WAIT_LIMIT = 1u << 22;


// Poll an mbarrier phase at most SCAN_WAIT_LIMIT times; false if it never completed.
__device__ __forceinline__ bool scan_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < SCAN_WAIT_LIMIT; ++i) {
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


// The chunk stream of one warp: items it0, it0 + stride, ...; each item's
// blocks [b0, b1) in chunks of cb blocks.
struct ChunkCursor {
    int64_t it;
    int c;  // chunk index within the item
};

template <int G, int SMAX, bool DIRECT, bool FULL>
__global__ void __launch_bounds__(SCAN_WARPS * 32, (SMAX <= 2 ? 3 : (SMAX <= 8 ? 2 : 1))) k_scan(ScanArgs A, ScanOut O, const int64_t* __restrict__ pair_off,
                                                          const int64_t* __restrict__ item_off,
                                                          const uint32_t* __restrict__ pairs, int L, int TB,
                                                          int32_t* __restrict__ status) {
    constexpr int QG = 32 / G;
    constexpr int V = 32 / G;
    constexpr bool SEL = scan_shared_sel<G>();
    constexpr int CHUNK = scan_chunk_bytes<G>();
    // SCAN_WARPS x 2 x CHUNK code buffers, then (SEL) SCAN_WARPS x M x 64 selector bytes
    extern __shared__ __align__(128) uint8_t bufs[];
    __shared__ __align__(8) uint64_t full[SCAN_WARPS][2];
    // kept keys of the warp's current item, per query slot, flushed to the
    // candidate store with one atomic per slot when a slot fills and when the
    // item ends (so a block's atomic latency is not on the scan's path)
    __shared__ uint64_t kbuf[SCAN_WARPS][QG][SCAN_BUF_KEYS];
    __shared__ int kcnt[SCAN_WARPS][QG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = lane / G, g = lane % G;
    constexpr bool direct = DIRECT;  // no threshold (O.thr null): keys to fixed places
    if (lane < QG) kcnt[warp][lane] = 0;
    const int M = A.M;
    const int S = (M + G - 1) / G;
    const int blk_bytes = M * 16;
    const int cb = CHUNK / blk_bytes;  // blocks per chunk (>= 1)
    const int64_t total = item_off[L];
    const int64_t stride = (int64_t)gridDim.x * SCAN_WARPS;
    uint8_t* mybuf = bufs + (size_t)warp * 2 * CHUNK;
    uint4* sel = reinterpret_cast<uint4*>(bufs + (size_t)SCAN_WARPS * 2 * CHUNK) + (size_t)warp * 4 * M;
    const uint32_t bar0 = smem_addr(&full[warp][0]), bar1 = smem_addr(&full[warp][1]);
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // lane 0: bulk copy of chunk (x, c) into buffer b
    auto issue = [&](const ScanItem& x, int c, int b) {
        const int c0 = x.b0 + c * cb, c1 = min(x.b1, c0 + cb);
        const uint32_t bytes = (uint32_t)(c1 - c0) * blk_bytes;
        const uint32_t bar = b ? bar1 : bar0;
        const uint8_t* src = A.codes + (A.boff[x.p] + c0) * (int64_t)blk_bytes;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_addr(mybuf + b * CHUNK)),
                     "l"(src), "r"(bytes), "r"(bar)
                     : "memory");
    };
    int64_t it = (int64_t)blockIdx.x * SCAN_WARPS + warp;
    if (it >= total) return;
    ScanItem x = locate_item(A, pair_off, item_off, L, TB, QG, it), nx = x;
    if (lane == 0) issue(x, 0, 0);
    uint32_t phase[2] = {0u, 0u};
    int b = 0;
    bool failed = false;
    while (true) {
        // item set-up: LUTs, bias and threshold of this lane group's query.
        // An item with fewer pairs than query slots (few queries probe the
        // list) gives every pair rep = QG / npw slots (npw: the pair count
        // rounded up to a power of two), which take interleaved blocks of each
        // chunk: slot = ph * npw + pi scans blocks ph, ph + rep, ...
        const int np_eff = (int)(x.npairs < QG ? x.npairs : QG);
        int npw = 1;
        while (npw < np_eff) npw <<= 1;
        const int rep = QG / npw;
        const int64_t pi = slot % npw;
        const int ph = slot / npw;
        const bool active = pi < np_eff;
        int64_t q = 0;
        uint4 t[SMAX];
        int32_t bias = 0, lim = -1;
        uint32_t thI = 0;
        int64_t noff = 0;
        if (active) {
            const uint32_t e = pairs[x.g0 + pi];
            q = e / A.Pmax;
            if (direct) noff = near_offset(A, q, (int)(e - q * A.Pmax));
            const uint4* lp = reinterpret_cast<const uint4*>(A.lut + (int64_t)e * M * PQ_K);
#pragma unroll
            for (int u = 0; u < SMAX; ++u) {
                const int j = g + G * u;
                t[u] = (FULL || (u < S && j < M)) ? __ldg(lp + j) : make_uint4(0, 0, 0, 0);
            }
            bias = A.bias[e];
            const uint64_t th = O.thr ? O.thr[q] : KEY_NONE;
            thI = (uint32_t)th;
            // key high word (bias + sum) + 2^31 vs the threshold's: sum < lim
            // passes, sum == lim is decided by the id (sums are below 2^24)
            const int64_t l = (int64_t)(th >> 32) - 2147483648ll - bias;
            lim = (int32_t)(l < -1 ? -1 : (l > (1 << 24) ? (1 << 24) : l));
        } else {
#pragma unroll
            for (int u = 0; u < SMAX; ++u) t[u] = make_uint4(0, 0, 0, 0);
        }
        // all lanes: each lane group writes its slot's buffered keys; a buffered
        // entry holds (distance word, vector slot in blk_ids), the id is
        // looked up here, many at once
        auto flush = [&]() {
            const int n = kcnt[warp][slot];
            int base = 0;
            if (g == 0 && n > 0) base = atomicAdd(&O.cnt[q], n);
            base = __shfl_sync(0xffffffffu, base, 0, G);
            for (int i0 = g; i0 < n; i0 += 4 * G) {  // four id loads in flight per lane
                uint64_t e[4];
                uint32_t id[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) e[u] = i0 + u * G < n ? kbuf[warp][slot][i0 + u * G] : 0ull;
#pragma unroll
                for (int u = 0; u < 4; ++u) id[u] = i0 + u * G < n ? (uint32_t)A.ids[(uint32_t)e[u]] : 0u;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * G;
                    if (i < n && base + i < O.cap) O.cand[q * O.cap + base + i] = (e[u] & 0xffffffff00000000ull) | id[u];
                }
            }
            __syncwarp();
            if (g == 0) kcnt[warp][slot] = 0;
            __syncwarp();
        };
        const int listn = A.list_n[x.p];
        const int nch = (x.b1 - x.b0 + cb - 1) / cb;
        const int64_t next_it = it + stride;
        for (int c = 0; c < nch; ++c) {
            // prefetch the chunk after this one into the other buffer
            if (c + 1 == nch && next_it < total) nx = locate_item(A, pair_off, item_off, L, TB, QG, next_it);
            if (lane == 0) {
                if (c + 1 < nch) issue(x, c + 1, b ^ 1);
                else if (next_it < total) issue(nx, 0, b ^ 1);
            }
            const bool ready = !failed && scan_wait(b ? bar1 : bar0, phase[b]);
            phase[b] ^= 1u;
            if (!ready) {
                if (lane == 0 && !failed) atomicOr(status, 4);  // a chunk never arrived: the warp stops
                failed = true;
            } else {
                const uint8_t* chunk = mybuf + b * CHUNK;
                const int c0 = x.b0 + c * cb, nblk = min(x.b1, c0 + cb) - c0;
                const int64_t gb0 = A.boff[x.p] + c0;
                // the same number of steps on every lane (the reduction is a
                // warp-wide shuffle); a slot past the chunk's last block reads
                // the last block again and keeps nothing
                for (int blk0 = 0; blk0 < nblk; blk0 += rep) {
                    const int blk = blk0 + ph;
                    const bool vb = active && blk < nblk;
                    const uint4* cp = reinterpret_cast<const uint4*>(chunk + min(blk, nblk - 1) * blk_bytes);
                    const uint32_t vslot = (uint32_t)((gb0 + blk) * 32 + V * g);
                    uint32_t idv[V];
                    if (direct && vb) {
#pragma unroll
                        for (int v = 0; v < V; ++v) idv[v] = (uint32_t)A.ids[vslot + v];
                    }
                    uint32_t a32[32];
#pragma unroll
                    for (int m = 0; m < 32; ++m) a32[m] = 0;
                    if (SEL && rep == 1) {
                        // every slot scans this block: its selectors once, into
                        // the warp's buffer (word k of subspace j at k M + j),
                        // then the lookups from there
                        for (int jj = lane; jj < M; jj += 32) {
                            const uint4 cw = cp[jj];
                            sel[0 * M + jj] = lut16_selectors(cw.x);
                            sel[1 * M + jj] = lut16_selectors(cw.y);
                            sel[2 * M + jj] = lut16_selectors(cw.z);
                            sel[3 * M + jj] = lut16_selectors(cw.w);
                        }
                        __syncwarp();
#pragma unroll
                        for (int u = 0; u + 1 < SMAX; u += 2) {
                            const int j = g + G * u;
                            if (FULL || (u + 1 < S && j + G < M)) accum_pair_sel(sel, M, j, j + G, t[u], t[u + 1], a32);
                            else if (u < S && j < M) accum_chunk_sel(sel, M, j, t[u], a32);
                        }
                        if (SMAX & 1) {
                            const int u = SMAX - 1, j = g + G * u;
                            if (FULL || (u < S && j < M)) accum_chunk_sel(sel, M, j, t[u], a32);
                        }
                        __syncwarp();  // all reads done before the next block's selectors
                    } else {
#pragma unroll
                        for (int u = 0; u + 1 < SMAX; u += 2) {
                            const int j = g + G * u;
                            if (FULL || (u + 1 < S && j + G < M)) accum_pair32(cp[j], t[u], cp[j + G], t[u + 1], a32);
                            else if (u < S && j < M) accum_chunk32(cp[j], t[u], a32);
                        }
                        if (SMAX & 1) {
                            const int u = SMAX - 1, j = g + G * u;
                            if (FULL || (u < S && j < M)) accum_chunk32(cp[j], t[u], a32);
                        }
                    }
                    // partial sums < 2^16: pack vector pairs for the reduction
                    uint32_t acc[16];
#pragma unroll
                    for (int m = 0; m < 16; ++m) acc[m] = prmt(a32[2 * m], a32[2 * m + 1], 0x5410u);
                    uint32_t sums[V];
                    reduce_scatter<G>(acc, lane, sums);
                    if (direct) {
                        if (vb) {
                            const int nv = listn - (c0 + blk) * 32;
                            const int64_t pos = noff + (int64_t)(c0 + blk) * 32 + V * g;
                            uint64_t* out = O.cand + q * O.cap;
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const uint32_t Dk = (uint32_t)(bias + (int32_t)sums[v]) ^ 0x80000000u;
                                if (V * g + v < nv && pos + v < O.cap) out[pos + v] = ((uint64_t)Dk << 32) | idv[v];
                            }
                        }
                        continue;
                    }
                    // keys at or below the threshold (padding, only at a list's
                    // tail, excluded by the list length); an id is read only
                    // on a tie with the threshold's distance
                    uint32_t kmask = 0;
                    if (vb) {
                        const int nv = listn - (c0 + blk) * 32 - V * g;  // valid vectors of this lane
                        const uint32_t vm = nv >= V ? (1u << V) - 1u : (nv > 0 ? (1u << nv) - 1u : 0u);
                        uint32_t eq = 0;
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            kmask |= (uint32_t)((int)sums[v] < lim) << v;
                            eq |= (uint32_t)((int)sums[v] == lim) << v;
                        }
                        kmask &= vm;
                        eq &= vm;
                        while (eq) {
                            const int v = __ffs(eq) - 1;
                            eq &= eq - 1u;
                            if ((uint32_t)A.ids[vslot + v] <= thI) kmask |= 1u << v;
                        }
                    }
                    // into the slot's buffer, which always has room for a whole
                    // block (32 keys): each lane reserves its keys with a shared
                    // atomic; a slot left with less room is flushed.  Entry:
                    // high word (D + 2^31) as an unsigned integer, low word the
                    // vector's slot (the id is looked up at the flush)
                    if (__any_sync(0xffffffffu, kmask != 0u)) {
                        if (kmask) {
                            const int pos = atomicAdd(&kcnt[warp][slot], __popc(kmask));
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                if ((kmask >> v) & 1u) {
                                    const uint32_t Dk = (uint32_t)(bias + (int32_t)sums[v]) ^ 0x80000000u;
                                    kbuf[warp][slot][pos + __popc(kmask & ((1u << v) - 1u))] =
                                        ((uint64_t)Dk << 32) | (vslot + v);
                                }
                        }
                        __syncwarp();
                        if (__any_sync(0xffffffffu, kcnt[warp][slot] > SCAN_BUF_KEYS - 32)) flush();
                    }
                }
            }
            __syncwarp();  // the whole warp is done with buffer b before lane 0 refills it
            b ^= 1;
        }
        if (__any_sync(0xffffffffu, kcnt[warp][slot] > 0)) flush();
        if (next_it >= total || failed) break;
        it = next_it;
        x = nx;
    }
}

// ------------------------------------------------------------------ a3: LUT16 scan, one lane per block
// Same warp items as k_scan with 4 lanes per query (list p, 8 queries that
// probe p, tile [b0, b1) of p's blocks), but the 4 lanes of a query take 4
// different blocks of each step and each sums all M subspaces of its block's
// 32 vectors, so no cross-lane reduction is needed.  Lane = (slot s = lane & 7,
// block bo = lane >> 3).  The item's 8 tables of subspace j sit side by side in
// shared memory (T[j][s], 16 B each): the 8 lanes of a quarter-warp (same bo,
// s = 0..7) read 128 contiguous bytes, and they share one block, so its code
// chunk is a broadcast.  Codes arrive in steps of 4 blocks by cp.async.bulk
// into two alternating buffers, as in k_scan.
constexpr int S4_WARPS = 4;
constexpr int S4_Q = 8;  // queries per item
constexpr int S4_B = 4;  // blocks per step

template <int MAXM>
__host__ __device__ constexpr int s4_warp_bytes() { return MAXM * S4_Q * 16 + 2 * S4_B * MAXM * 16; }

template <int MAXM>
__global__ void __launch_bounds__(S4_WARPS * 32, MAXM <= 64 ? 3 : 1)
    k_scan4(ScanArgs A, ScanOut O, const int64_t* __restrict__ pair_off, const int64_t* __restrict__ item_off,
            const uint32_t* __restrict__ pairs, int L, int TB, int32_t* __restrict__ status) {
    constexpr int TAB_BYTES = MAXM * S4_Q * 16;
    constexpr int BUF_BYTES = S4_B * MAXM * 16;
    extern __shared__ __align__(128) uint8_t sm4[];
    __shared__ __align__(8) uint64_t full[S4_WARPS][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = lane & 7, bo = lane >> 3;
    const int M = A.M, blk_bytes = M * 16;
    const bool direct = O.thr == nullptr;
    uint8_t* wb = sm4 + (size_t)warp * s4_warp_bytes<MAXM>();
    uint4* tab = reinterpret_cast<uint4*>(wb);
    uint8_t* cbuf = wb + TAB_BYTES;
    const uint32_t bar0 = smem_addr(&full[warp][0]), bar1 = smem_addr(&full[warp][1]);
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    auto issue = [&](const ScanItem& x, int c, int b) {
        const int c0 = x.b0 + c * S4_B, c1 = min(x.b1, c0 + S4_B);
        const uint32_t bytes = (uint32_t)(c1 - c0) * blk_bytes;
        const uint32_t bar = b ? bar1 : bar0;
        const uint8_t* src = A.codes + (A.boff[x.p] + c0) * (int64_t)blk_bytes;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_addr(cbuf + b * BUF_BYTES)),
                     "l"(src), "r"(bytes), "r"(bar)
                     : "memory");
    };
    const int64_t total = item_off[L];
    const int64_t stride = (int64_t)gridDim.x * S4_WARPS;
    int64_t it = (int64_t)blockIdx.x * S4_WARPS + warp;
    if (it >= total) return;
    ScanItem x = locate_item(A, pair_off, item_off, L, TB, S4_Q, it, S4_B), nx = x;
    if (lane == 0) issue(x, 0, 0);
    uint32_t phase[2] = {0u, 0u};
    int b = 0;
    bool failed = false;
    while (true) {
        // the item's tables, transposed to T[j][s] (zeros for empty slots)
        const int nslots = x.npairs < S4_Q ? (int)x.npairs : S4_Q;
        for (int e = lane; e < S4_Q * M; e += 32) {
            const int qs = e / M, j = e - qs * M;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (qs < nslots) v = __ldg(reinterpret_cast<const uint4*>(A.lut + (int64_t)pairs[x.g0 + qs] * M * PQ_K) + j);
            tab[j * S4_Q + qs] = v;
        }
        const bool active = s < nslots;
        int64_t q = 0, noff = 0;
        int32_t bias = 0, lim = -1;
        uint32_t thI = 0;
        if (active) {
            const uint32_t e = pairs[x.g0 + s];
            q = e / A.Pmax;
            if (direct) noff = near_offset(A, q, (int)(e - q * A.Pmax));
            bias = A.bias[e];
            const uint64_t th = O.thr ? O.thr[q] : KEY_NONE;
            thI = (uint32_t)th;
            // key high word (bias + sum) + 2^31 <= thD  <=>  sum <= thD - 2^31 - bias
            const int64_t l = (int64_t)(th >> 32) - 2147483648ll - bias;
            lim = (int32_t)(l < -1 ? -1 : (l > 65536 ? 65536 : l));
        }
        const int listn = A.list_n[x.p];
        const int64_t gb_list = A.boff[x.p];
        __syncwarp();
        const int nch = (x.b1 - x.b0 + S4_B - 1) / S4_B;
        const int64_t next_it = it + stride;
        for (int c = 0; c < nch; ++c) {
            if (c + 1 == nch && next_it < total) nx = locate_item(A, pair_off, item_off, L, TB, S4_Q, next_it, S4_B);
            if (lane == 0) {
                if (c + 1 < nch) issue(x, c + 1, b ^ 1);
                else if (next_it < total) issue(nx, 0, b ^ 1);
            }
            const bool ready = !failed && scan_wait(b ? bar1 : bar0, phase[b]);
            phase[b] ^= 1u;
            if (!ready) {
                if (lane == 0 && !failed) atomicOr(status, 4);  // a chunk never arrived: the warp stops
                failed = true;
            } else {
                const int c0 = x.b0 + c * S4_B, nblk = min(x.b1, c0 + S4_B) - c0;
                const int blk = c0 + bo;
                uint32_t acc[32];  // sum of vector v of the block
#pragma unroll
                for (int m = 0; m < 32; ++m) acc[m] = 0u;
                uint32_t kmask = 0;
                if (bo < nblk) {
                    const uint4* cp = reinterpret_cast<const uint4*>(cbuf + b * BUF_BYTES + bo * blk_bytes);
                    const uint4* tp = tab + s;
                    int j = 0;
                    for (; j + 1 < M; j += 2) accum_pair32(cp[j], tp[j * S4_Q], cp[j + 1], tp[(j + 1) * S4_Q], acc);
                    if (j < M) accum_chunk32(cp[j], tp[j * S4_Q], acc);
                    if (direct && active) {
                        // no threshold: every key of the block to its fixed place
                        const int nv = listn - blk * 32;
                        const int64_t pos = noff + (int64_t)blk * 32;
                        const int32_t* idp = A.ids + (gb_list + blk) * 32;
                        uint64_t* out = O.cand + q * O.cap;
#pragma unroll
                        for (int v = 0; v < 32; ++v) {
                            const uint32_t Dk = (uint32_t)(bias + (int32_t)acc[v]) ^ 0x80000000u;
                            if (v < nv && pos + v < O.cap) out[pos + v] = ((uint64_t)Dk << 32) | (uint32_t)idp[v];
                        }
                    } else if (active) {
                        const int nv = listn - blk * 32;
                        const uint32_t vmask = nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u);
                        uint32_t lt = 0, eq = 0;
#pragma unroll
                        for (int v = 0; v < 32; ++v) {
                            lt |= (uint32_t)((int)acc[v] < lim) << v;
                            eq |= (uint32_t)((int)acc[v] == lim) << v;
                        }
                        lt &= vmask;
                        eq &= vmask;
                        while (eq) {  // a key equal to the threshold's distance: its id decides
                            const int v = __ffs(eq) - 1;
                            eq &= eq - 1u;
                            if ((uint32_t)A.ids[(gb_list + blk) * 32 + v] <= thI) lt |= 1u << v;
                        }
                        kmask = lt;
                    }
                }
                // one atomic per query and step: counts of its 4 lanes (kmask
                // stays empty with no threshold: those keys are already placed)
                const int n = __popc(kmask);
                const int n0 = __shfl_sync(0xffffffffu, n, s), n1 = __shfl_sync(0xffffffffu, n, s + 8);
                const int n2 = __shfl_sync(0xffffffffu, n, s + 16), n3 = __shfl_sync(0xffffffffu, n, s + 24);
                const int tot = n0 + n1 + n2 + n3;
                int base = (bo == 0 && tot > 0) ? atomicAdd(&O.cnt[q], tot) : 0;
                base = __shfl_sync(0xffffffffu, base, s) + (bo > 0 ? n0 : 0) + (bo > 1 ? n1 : 0) + (bo > 2 ? n2 : 0);
                if (kmask) {
                    const int32_t* idp = A.ids + (gb_list + blk) * 32;
                    uint64_t* out = O.cand + q * O.cap;
#pragma unroll
                    for (int v = 0; v < 32; ++v) {
                        if ((kmask >> v) & 1u) {
                            const int at = base + __popc(kmask & ((1u << v) - 1u));
                            const uint32_t Dk = (uint32_t)(bias + (int32_t)acc[v]) ^ 0x80000000u;
                            if (at < O.cap) out[at] = ((uint64_t)Dk << 32) | (uint32_t)idp[v];
                        }
                    }
                }
            }
            __syncwarp();  // the whole warp is done with buffer b (and the tables) before they are refilled
            b ^= 1;
        }
        if (next_it >= total || failed) break;
        it = next_it;
        x = nx;
    }
}

// ------------------------------------------------------------------ a4: hybrid graph search
// Work lists from an explicit pair array (the lists marked for a full scan).
__global__ void k_count_from(const uint32_t* __restrict__ src, const int64_t* __restrict__ nsrc,
                             const int32_t* __restrict__ probes, int32_t* __restrict__ cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= *nsrc) return;
    atomicAdd(&cnt[probes[src[i]]], 1);
}

__global__ void k_fill_from(const uint32_t* __restrict__ src, const int64_t* __restrict__ nsrc,
                            const int32_t* __restrict__ probes, const int64_t* __restrict__ pair_off,
                            int32_t* __restrict__ fill, uint32_t* __restrict__ dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= *nsrc) return;
    const uint32_t e = src[i];
    const int p = probes[e];
    dst[pair_off[p] + atomicAdd(&fill[p], 1)] = e;
}

struct GraphArgs {
    const int32_t* nbr_pos;    // [nslots x 32] neighbour list positions, -1 padding
    const uint8_t* nbr_codes;  // [nslots x M x 16] neighbour codes as one block per node
    const int32_t* entry_pos;  // [L]
    int efs, tau, vwords;
    uint32_t* full_pairs;      // out: (query, rank) pairs whose list is scanned fully
    int64_t* nfull;            // out: their count
};

constexpr int GS_WARPS = 4;
constexpr int GS_N = 128;  // W (<= efs <= 96) plus 32 new keys, sorted together

// 32 distances of one block for the lane group of the whole warp (G = 32):
// lane l receives vector l's sum.
template <int SMAX>
__device__ __forceinline__ uint32_t block_sums32(const uint4* __restrict__ cp, const uint4 (&t)[SMAX], int M,
                                                 int lane) {
    uint32_t acc[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) acc[m] = 0;
#pragma unroll
    for (int u = 0; u < SMAX; ++u) {
        const int j = lane + 32 * u;
        if (j < M) accum_chunk(__ldg(cp + j), t[u], acc);
    }
    uint32_t out[1];
    reduce_scatter<32>(acc, lane, out);
    return out[0];
}

// One warp per (query, distant list): best-first search of the list's graph
// with result set W of capacity efs (Sec. 4.4).  W is kept sorted in shared
// memory with, per entry, its list position and whether it was expanded; an
// expansion takes the smallest unexpanded entry, computes its 32
// neighbours' keys with one LUT16 block, marks them visited, and keeps the
// efs smallest of W and the unvisited neighbours.  The search ends when every
// entry of W is expanded (equivalently: the best candidate is worse than
// W's worst once W is full).  Then, with theta the query's threshold: at
// least tau keys of W below theta -> the list is scanned fully later;
// otherwise W's keys at or below theta join the candidates.
template <int SMAX>
__global__ void __launch_bounds__(GS_WARPS * 32) k_graph_search(ScanArgs A, ScanOut O, GraphArgs Gr,
                                                                const uint32_t* __restrict__ pairs,
                                                                const int64_t* __restrict__ npairs) {
    extern __shared__ __align__(16) uint8_t gsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t per_warp = (size_t)GS_N * 16 + (size_t)Gr.vwords * 4;
    uint8_t* base_w = gsm + warp * per_warp;
    uint64_t* wk = reinterpret_cast<uint64_t*>(base_w);             // keys
    int32_t* wp = reinterpret_cast<int32_t*>(base_w + GS_N * 8);    // list positions
    uint32_t* wf = reinterpret_cast<uint32_t*>(base_w + GS_N * 12); // expanded flags
    uint32_t* vis = reinterpret_cast<uint32_t*>(base_w + GS_N * 16);
    const int M = A.M;
    const int64_t n_items = *npairs;
    for (int64_t it = (int64_t)blockIdx.x * GS_WARPS + warp; it < n_items; it += (int64_t)gridDim.x * GS_WARPS) {
        const uint32_t e = pairs[it];
        const int64_t q = e / A.Pmax;
        const int p = A.probes[e];
        const int np_ = A.list_n[p];
        const int ep = Gr.entry_pos[p];
        if (ep < 0) continue;
        uint4 t[SMAX];
        const uint4* lp = reinterpret_cast<const uint4*>(A.lut + (int64_t)e * M * PQ_K);
#pragma unroll
        for (int u = 0; u < SMAX; ++u) {
            const int j = lane + 32 * u;
            t[u] = j < M ? __ldg(lp + j) : make_uint4(0, 0, 0, 0);
        }
        const int32_t bias = A.bias[e];
        const uint64_t th = O.thr[q];
        const int64_t slot0 = A.boff[p] * 32;
        for (int w = lane; w < (np_ + 31) / 32; w += 32) vis[w] = 0u;
        __syncwarp();
        // entry: its block's 32 sums, keep the entry's
        {
            const int64_t gb = A.boff[p] + (ep >> 5);
            const uint32_t sum = block_sums32<SMAX>(reinterpret_cast<const uint4*>(A.codes + gb * M * 16), t, M, lane);
            if (lane == (ep & 31)) {
                wk[0] = make_key(bias + (int32_t)sum, A.ids[slot0 + ep]);
                wp[0] = ep;
                wf[0] = 0;
                vis[ep >> 5] = 1u << (ep & 31);
            }
            __syncwarp();
        }
        int wn = 1;
        for (int guard = 0; guard <= np_; ++guard) {
            // smallest unexpanded entry of the sorted W
            int ui = -1;
            for (int c = 0; c < wn && ui < 0; c += 32) {
                const bool un = (c + lane < wn) && wf[c + lane] == 0;
                const unsigned b = __ballot_sync(0xffffffffu, un);
                if (b) ui = c + __ffs(b) - 1;
            }
            if (ui < 0) break;
            const int upos = wp[ui];
            __syncwarp();
            if (lane == 0) wf[ui] = 1;
            // expand: the 32 neighbours' keys in one block
            const int64_t su = slot0 + upos;
            const uint32_t sum =
                block_sums32<SMAX>(reinterpret_cast<const uint4*>(Gr.nbr_codes + su * M * 16), t, M, lane);
            const int pe = Gr.nbr_pos[su * 32 + lane];
            uint64_t kn = KEY_NONE;
            if (pe >= 0) {
                const uint32_t bit = 1u << (pe & 31);
                const uint32_t old = atomicOr(&vis[pe >> 5], bit);
                if (!(old & bit)) kn = make_key(bias + (int32_t)sum, A.ids[slot0 + pe]);
            }
            wk[wn + lane] = kn;
            wp[wn + lane] = pe;
            wf[wn + lane] = 0;
            // sort W and the new keys together; keep the efs smallest
            const int N = wn + 32;
            const int S = N <= 64 ? 64 : GS_N;
            for (int i = N + lane; i < S; i += 32) wk[i] = KEY_NONE;
            __syncwarp();
            for (int k2 = 2; k2 <= S; k2 <<= 1)
                for (int j = k2 >> 1; j > 0; j >>= 1) {
                    for (int i = lane; i < S; i += 32) {
                        const int ixj = i ^ j;
                        if (ixj > i) {
                            const uint64_t a = wk[i], b2 = wk[ixj];
                            const bool up = (i & k2) == 0;
                            if ((a > b2) == up) {
                                wk[i] = b2;
                                wk[ixj] = a;
                                const int32_t tp = wp[i];
                                wp[i] = wp[ixj];
                                wp[ixj] = tp;
                                const uint32_t tf = wf[i];
                                wf[i] = wf[ixj];
                                wf[ixj] = tf;
                            }
                        }
                    }
                    __syncwarp();
                }
            int valid = 0;
            for (int c = 0; c < S; c += 32) valid += __popc(__ballot_sync(0xffffffffu, c + lane < S && wk[c + lane] != KEY_NONE));
            wn = min(valid, Gr.efs);
        }
        // decide: full scan later, or W's keys join the candidates
        int good = 0;
        for (int c = 0; c < wn; c += 32) good += __popc(__ballot_sync(0xffffffffu, c + lane < wn && wk[c + lane] < th));
        if (good >= Gr.tau) {
            if (lane == 0) Gr.full_pairs[atomicAdd(reinterpret_cast<unsigned long long*>(Gr.nfull), 1ull)] = e;
        } else {
            for (int c = 0; c < wn; c += 32) {
                const bool keep = c + lane < wn && wk[c + lane] <= th;
                const unsigned b = __ballot_sync(0xffffffffu, keep);
                int base = 0;
                if (lane == 0 && b) base = atomicAdd(&O.cnt[q], __popc(b));
                base = __shfl_sync(0xffffffffu, base, 0) + __popc(b & ((1u << lane) - 1u));
                if (keep && base < O.cap) O.cand[q * O.cap + base] = wk[c + lane];
            }
        }
        __syncwarp();
    }
}

// The scan's lookup sequence with shared selectors (8 lanes per query): the
// selectors of a subspace pair from the warp's shared buffer (at indices that
// depend on a per-iteration random number, so that nothing can be hoisted
// out of the loop), the lookups and the interleaved widening of two
// subspaces -- the lookup rate of the scan's inner loop with no code or
// table traffic beyond shared memory.
__global__ void __launch_bounds__(256) k_lut16_peak_sel(int iters, uint32_t seed, uint32_t* __restrict__ sink) {
    __shared__ uint4 sel[4 * 64];
    for (int i = threadIdx.x; i < 4 * 64; i += blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u + seed;
        h ^= h >> 15;
        h *= 0x2c1b3c6du;
        sel[i] = lut16_selectors(h ^ (h >> 12));
    }
    __syncthreads();
    const int g = threadIdx.x & 7;
    const uint4 t0 = make_uint4(seed, seed * 3u + 1u, seed * 5u + 7u, seed * 9u + 3u);
    const uint4 t1 = make_uint4(t0.y, t0.z, t0.w, t0.x);
    uint32_t acc[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) acc[m] = 0;
    uint32_t w = seed ^ (blockIdx.x * blockDim.x + threadIdx.x);
    for (int i = 0; i < iters; i += 2) {  // 64 lookups per pair of iterations
        const int j = (g + 8 * (int)(w >> 29)) & 63;
        accum_pair_sel(sel, 64, j, (j + 32) & 63, t0, t1, acc);
        w = w * 1664525u + 1013904223u;
    }
    uint32_t s_ = 0;
#pragma unroll
    for (int m = 0; m < 32; ++m) s_ ^= acc[m];
    if (s_ == 0x12345678u) sink[0] = s_;  // keeps the loop alive
}

// Register-only copy of the scan's earlier lookup/accumulate sequence (each
// query slot computing its own selectors, one byte dot product per lookup;
// no memory traffic): still the sequence of the scan's sparse items.
__global__ void __launch_bounds__(128) k_lut16_peak(int iters, uint32_t seed, uint32_t* __restrict__ sink) {
    uint4 t = make_uint4(seed, seed * 3u + 1u, seed * 5u + 7u, seed * 9u + 3u);
    uint32_t acc[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) acc[m] = 0;
    uint32_t w = seed ^ (blockIdx.x * blockDim.x + threadIdx.x);
    const uint4 t2 = make_uint4(t.y, t.z, t.w, t.x);
    for (int i = 0; i < iters; i += 2) {
        uint4 c = make_uint4(w, w ^ 0x5a5a5a5au, w + 0x01234567u, w ^ 0xf0f0f0f0u);
        uint4 c2 = make_uint4(w ^ 0x0f0f0f0fu, w + 0x89abcdefu, w ^ 0x33333333u, w + 0x13579bdfu);
        accum_pair32(c, t, c2, t2, acc);
        w = w * 1664525u + 1013904223u;
    }
    uint32_t s = 0;
#pragma unroll
    for (int m = 0; m < 32; ++m) s ^= acc[m];
    if (s == 0x12345678u) sink[0] = s;  // keeps the loop alive
}

// ------------------------------------------------------------------ a5: select
// R smallest candidate keys per query, in no particular order (the re-rank
// does not need one); one warp per query.  A query whose store overflowed is
// put on the redo list for k_select_redo.
__global__ void __launch_bounds__(SW_WARPS * 32) k_select(ScanArgs A, int Rmax, const int32_t* __restrict__ cnt,
                                                          const uint64_t* __restrict__ cand, int cap,
                                                          uint64_t* __restrict__ topr, int32_t* __restrict__ ncand,
                                                          int32_t* __restrict__ status,
                                                          unsigned long long* __restrict__ stats,
                                                          int32_t* __restrict__ redo) {
    __shared__ uint32_t hist[SW_WARPS][256];
    __shared__ uint64_t bb[SW_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * SW_WARPS + w;
    if (q >= A.nq) return;
    const int R = rerank_of(A.rerank_q, A.Rfix, A.Rmin, Rmax, q);
    const int n = cnt[q];
    if (lane == 0) {
        atomicAdd(&stats[1], (unsigned long long)n);
        atomicMax(&stats[2], (unsigned long long)n);
    }
    if (n > cap) {
        if (lane == 0) {
            atomicAdd(&stats[0], 1ull);
            atomicOr(status, KSC_STATUS_CAND_OVERFLOW);
            redo[1 + atomicAdd(&redo[0], 1)] = (int32_t)q;
        }
        return;
    }
    const uint64_t* cq = cand + q * cap;
    uint64_t* out = topr + q * Rmax;
    const int K = min(R, n);
    if (n <= K) {
        for (int i = lane; i < n; i += 32) out[i] = cq[i];
    } else {
        warp_topk_hi(cq, n, K, out, hist[w], bb[w]);
    }
    for (int i = K + lane; i < Rmax; i += 32) out[i] = KEY_NONE;
    if (lane == 0 && ncand) ncand[q] = K;
}

// The same with one CTA per query, for queries with many candidates.
template <int NT>
__global__ void __launch_bounds__(NT) k_select_cta(ScanArgs A, int Rmax, const int32_t* __restrict__ cnt,
                                                    const uint64_t* __restrict__ cand, int cap,
                                                    uint64_t* __restrict__ topr, int32_t* __restrict__ ncand,
                                                    int32_t* __restrict__ status,
                                                    unsigned long long* __restrict__ stats,
                                                    int32_t* __restrict__ redo) {
    __shared__ uint32_t hist[256];
    __shared__ uint64_t bb[32];
    const int64_t q = blockIdx.x;
    const int R = rerank_of(A.rerank_q, A.Rfix, A.Rmin, Rmax, q);
    const int n = cnt[q];
    if (threadIdx.x == 0) {
        atomicAdd(&stats[1], (unsigned long long)n);
        atomicMax(&stats[2], (unsigned long long)n);
    }
    if (n > cap) {
        if (threadIdx.x == 0) {
            atomicAdd(&stats[0], 1ull);
            atomicOr(status, KSC_STATUS_CAND_OVERFLOW);
            redo[1 + atomicAdd(&redo[0], 1)] = (int32_t)q;
        }
        return;
    }
    const uint64_t* cq = cand + q * cap;
    uint64_t* out = topr + q * Rmax;
    const int K = min(R, n);
    if (n <= K) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = cq[i];
    } else {
        auto load = [&](int i) -> uint64_t { return cq[i]; };
        auto emit = [&](int i, uint64_t k) { out[i] = k; };
        block_topk(load, n, K, emit, hist, bb);
    }
    for (int i = K + threadIdx.x; i < Rmax; i += blockDim.x) out[i] = KEY_NONE;
    if (threadIdx.x == 0 && ncand) ncand[q] = K;
}

// Queries whose candidate store overflowed, redone exactly: every key of every
// probed list is recomputed (scalar lookups) inside the radix select.  A
// persistent grid walks the redo list (usually empty).
__global__ void __launch_bounds__(256) k_select_redo(ScanArgs A, int Rmax, int sel_cap, uint64_t* __restrict__ topr,
                                                     int32_t* __restrict__ ncand, const int32_t* __restrict__ redo) {
    extern __shared__ uint64_t sbuf[];  // sel_cap keys
    __shared__ uint32_t hist[256];
    __shared__ int32_t s_pref[MAX_NPROBE + 1];
    const int nredo = redo[0];
    for (int r0 = blockIdx.x; r0 < nredo; r0 += gridDim.x) {
        const int64_t q = redo[1 + r0];
        const int R = rerank_of(A.rerank_q, A.Rfix, A.Rmin, Rmax, q);
        uint64_t* out = topr + q * Rmax;
        const int P = nprobe_of(A, q);
        __syncthreads();  // s_pref of the previous query is no longer read
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int r = 0; r < P; ++r) {
                s_pref[r] = acc;
                const int p = A.probes[q * A.Pmax + r];
                acc += (p >= 0 && p < A.L) ? A.list_n[p] : 0;
            }
            s_pref[P] = acc;
        }
        __syncthreads();
        const int N = s_pref[P];
        auto load = [&](int i) -> uint64_t {
            int lo = 0, hi = P - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (s_pref[mid] <= i) lo = mid; else hi = mid - 1;
            }
            const int64_t item = q * A.Pmax + lo;
            const int p = A.probes[item];
            const int m = i - s_pref[lo];
            const int64_t blk = A.boff[p] + (m >> 5);
            const int v = m & 31;
            int32_t D = scalar_dist(A.lut + item * A.M * PQ_K, A.bias[item], A.codes + blk * A.M * 16, A.M, v);
            return make_key(D, A.ids[blk * 32 + v]);
        };
        const int K = min(R, N);
        block_select_smallest(load, N, K, out, sbuf, sel_cap, hist);
        for (int i = K + threadIdx.x; i < Rmax; i += blockDim.x) out[i] = KEY_NONE;
        if (threadIdx.x == 0 && ncand) ncand[q] = K;
    }
}

// ------------------------------------------------------------------ a6: rerank
// Exact distance of each candidate (warp per candidate, 16-byte loads when d
// is a multiple of 4): L2 = sum (q_t - x_t)^2, IP = -<q, x>; the k best by
// (distance, id).  Output: L2 distance ascending / IP similarity descending.
template <int NT>
__global__ void __launch_bounds__(NT) k_rerank(const float* __restrict__ Q, const float* __restrict__ X, int d,
                                                int ip, const uint64_t* __restrict__ topr, int Rmax,
                                                const int32_t* __restrict__ rerank_q, int Rfix, int k,
                                                int64_t* __restrict__ out_ids, float* __restrict__ out_d) {
    extern __shared__ uint64_t keys[];
    __shared__ __align__(16) float qs[KSC_MAX_DIM];
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int R = rerank_of(rerank_q, Rfix, k, Rmax, q);
    for (int t = threadIdx.x; t < d; t += blockDim.x) qs[t] = Q[q * d + t];
    // the candidate keys staged in shared memory (each row load then waits
    // for a shared load); each slot is later replaced by its FP32 key by
    // the one warp that read it
    for (int c = threadIdx.x; c < R; c += blockDim.x) keys[c] = topr[q * Rmax + c];
    __syncthreads();
    const uint64_t* cq = keys;
    const bool vec4 = (d & 3) == 0;
    if (vec4 && d <= 128) {
        // one float4 per lane per row; four rows in flight per warp
        const bool inl = lane * 4 < d;
        const float4 qv = inl ? *reinterpret_cast<const float4*>(qs + lane * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c0 = w * 4; c0 < R; c0 += nw * 4) {
            float4 xv[4];
            int32_t idv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t kk = c0 + u < R ? cq[c0 + u] : KEY_NONE;
                idv[u] = kk != KEY_NONE ? (int32_t)(kk & 0xffffffffu) : -1;
                xv[u] = (idv[u] >= 0 && inl) ? __ldg(reinterpret_cast<const float4*>(X + (int64_t)idv[u] * d) + lane)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                float s = 0.f;
                if (ip) {
                    s = qv.x * xv[u].x + qv.y * xv[u].y + qv.z * xv[u].z + qv.w * xv[u].w;
                } else {
                    const float e0 = qv.x - xv[u].x, e1 = qv.y - xv[u].y, e2 = qv.z - xv[u].z, e3 = qv.w - xv[u].w;
                    s = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, e3 * e3)));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                __syncwarp();  // (every lane read the step's keys before they are replaced)
                if (lane == 0 && c0 + u < R)
                    keys[c0 + u] = idv[u] >= 0 ? (((uint64_t)ordered_f32(ip ? -s : s) << 32) | (uint32_t)idv[u])
                                               : KEY_NONE;
            }
        }
    } else
    for (int c = w; c < R; c += nw) {
        const uint64_t kk = cq[c];
        uint64_t outk = KEY_NONE;
        if (kk != KEY_NONE) {
            const int32_t id = (int32_t)(kk & 0xffffffffu);
            const float* x = X + (int64_t)id * d;
            float s = 0.f;
            if (vec4) {
                for (int t = lane * 4; t < d; t += 128) {
                    float4 xv = __ldg(reinterpret_cast<const float4*>(x + t));
                    float4 qv = *reinterpret_cast<const float4*>(qs + t);
                    if (ip) {
                        s = fmaf(qv.x, xv.x, s); s = fmaf(qv.y, xv.y, s);
                        s = fmaf(qv.z, xv.z, s); s = fmaf(qv.w, xv.w, s);
                    } else {
                        float e0 = qv.x - xv.x, e1 = qv.y - xv.y, e2 = qv.z - xv.z, e3 = qv.w - xv.w;
                        s = fmaf(e0, e0, s); s = fmaf(e1, e1, s); s = fmaf(e2, e2, s); s = fmaf(e3, e3, s);
                    }
                }
            } else {
                for (int t = lane; t < d; t += 32) {
                    float xv = __ldg(x + t);
                    if (ip) s = fmaf(qs[t], xv, s);
                    else { float e = qs[t] - xv; s = fmaf(e, e, s); }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const float dist = ip ? -s : s;
            outk = ((uint64_t)ordered_f32(dist) << 32) | (uint32_t)id;
        }
        __syncwarp();  // (every lane read the key before it is replaced)
        if (lane == 0) keys[c] = outk;
    }
    __syncthreads();
    if (k <= 32) {
        // k rounds of a warp minimum over the R keys (each taken key is retired)
        if (w == 0) {
            uint64_t mine = KEY_NONE;  // lane r keeps the r-th smallest
            for (int r = 0; r < k; ++r) {
                uint64_t m = KEY_NONE;
                int at = -1;
                for (int i = lane; i < R; i += 32) {
                    if (keys[i] < m) { m = keys[i]; at = i; }
                }
                uint64_t g = m;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const uint64_t y = __shfl_xor_sync(0xffffffffu, g, o);
                    g = y < g ? y : g;
                }
                if (g != KEY_NONE && m == g) keys[at] = KEY_NONE;  // keys are unique: one lane matches
                __syncwarp();
                if (lane == r) mine = g;
            }
            if (lane < k) keys[lane] = mine;
        }
        __syncthreads();
    } else {
        const int S = pow2_ceil(R < 2 ? 2 : R);
        for (int i = R + threadIdx.x; i < S; i += blockDim.x) keys[i] = KEY_NONE;
        __syncthreads();
        block_bitonic_sort(keys, S);
    }
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        const uint64_t kk = r < R ? keys[r] : KEY_NONE;
        if (kk == KEY_NONE) {
            out_ids[q * k + r] = -1;
            out_d[q * k + r] = ip ? -INFINITY : INFINITY;
        } else {
            out_ids[q * k + r] = (int64_t)(kk & 0xffffffffu);
            const float dist = unordered_f32((uint32_t)(kk >> 32));
            out_d[q * k + r] = ip ? -dist : dist;
        }
    }
}

// One warp per query (8 per CTA) when k <= 32, R <= RW_MAXR, d <= 128 and
// d % 4 == 0: lane l holds query coordinates 4l..4l+3; each step gathers 8
// candidate rows (one 16-byte load per lane and row) and sums the 8 partial
// dot products across the warp in a halving exchange (9 shuffles for 8 rows);
// the k best keys are then taken by k rounds of a warp minimum.  Same
// distance rule as k_rerank (L2 direct difference squares, IP -<q, x>), FP32.
//
// With xb (BF16 copies of the rows; or xu, U8 copies, when every coordinate
// is an integer in [0, 255] and a byte holds it exactly) and xe (per row:
// n >= |x| and r >= |x~ - x|, the norm of its rounding error, both from FP64
// sums rounded up), a first pass reads the low-precision rows (half or a
// quarter of the bytes) and bounds
// each candidate's FP32 distance: |d~ - d| <= e, from the rounding of the row
// (|<v, x~ - x>| <= |v| r) and the FP32 evaluation of both sums (relative
// g = 2^-20, above the at most 14 rounding steps of 2^-24 on a term's path in
// either pass):
//   L2: e = 2 r s + r^2 + g (s^2 + (s + r)^2), s >= sqrt of the exact
//       BF16-row distance (so s + r >= |q - x|);
//   IP: e = |q| (r + 2.01 g (n + r)),
// all evaluated with a factor (1 + 2^-10) and directed rounding of d~ -/+ e.
// r is the row's own rounding error, not the format's worst case
// (2^-8 |x|): a row that BF16 holds exactly (integer coordinates up to 256,
// say) has r = 0 and a band of the evaluation term alone.  U is the k-th
// smallest d~ + e; a candidate with d~ - e > U has an FP32 distance above k
// FP32 distances, so it cannot be among the k best.  The others get the FP32
// distance by the very code of the plain pass (a row's sum does not depend on
// the rows beside it in the exchange), so the result is bit for bit the
// plain pass's.
constexpr int RW_WARPS = 8;
constexpr int RW_MAXR = 512;

// Halving exchange of 8 rows' partial sums over the warp (9 shuffles):
// afterwards every lane of quad `myrow` (lane bits 4, 3, 2) holds that row's
// total, summed in the same tree for every row.
__device__ __forceinline__ float exchange_rows8(float (&a)[8], int lane) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 16;
        const float send = up ? a[i] : a[i + 4], keep = up ? a[i + 4] : a[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 8;
        const float send = up ? a[i] : a[i + 2], keep = up ? a[i + 2] : a[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const bool up = lane & 4;
        const float send = up ? a[0] : a[1], keep = up ? a[1] : a[0];
        a[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 2);
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
    return a[0];
}

// FP32 partial sums of the 8 rows idv[] (-1: none) for this lane's 4
// coordinates, summed across the warp: every lane of quad `myrow` ends with
// that row's distance term (L2: the squared distance, IP: the dot product).
__device__ __forceinline__ float rerank_rows8(const float4& qv, const float* __restrict__ X, int d, int ip, bool inl,
                                              const int32_t (&idv)[8], int lane) {
    float4 xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
        xv[u] = (idv[u] >= 0 && inl) ? __ldg(reinterpret_cast<const float4*>(X + (int64_t)idv[u] * d) + lane)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
    float a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        if (ip) {
            a[u] = qv.x * xv[u].x + qv.y * xv[u].y + qv.z * xv[u].z + qv.w * xv[u].w;
        } else {
            const float e0 = qv.x - xv[u].x, e1 = qv.y - xv[u].y, e2 = qv.z - xv[u].z, e3 = qv.w - xv[u].w;
            a[u] = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, e3 * e3)));
        }
    }
    return exchange_rows8(a, lane);
}

// The distance terms of 16 low-precision rows at once, 8 lanes per row:
// lane l = 8 h + j takes rows 4 h .. 4 h + 3 of the step (idv[], -1: none)
// and, of each, the 4-coordinate chunks j, j + 8, j + 16, j + 24 below d (one
// load each: 8 bytes of BF16, or 4 bytes of U8 rows; qv[] holds the query's
// coordinates of those chunks), summed in FP32 pairs; a halving exchange over
// lane bits 2, 1 and a sum over bit 0 leave row (lane >> 1) & 15 in both
// lanes of a pair.  The row's id, address and exchange cost one lane in
// eight, not every lane.  Only bounded, not compared bit for bit, so the
// summation order is free (its depth, at most 8 + 1 + 3 additions after the
// square, stays inside the bound's g).  A U8 byte b becomes the float
// (2^23 + b) - 2^23, exact.
template <bool U8>
__device__ __forceinline__ float rerank_rows16_band(const float4 (&qv)[4], const void* __restrict__ rows, int d,
                                                    int ip, int nch, const int32_t (&idv)[4], int lane) {
    const int j = lane & 7;
    uint2 r[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = k < nch && idv[i] >= 0 && 4 * (j + 8 * k) < d;
            if (U8)
                r[i][k] = make_uint2(ok ? __ldg(reinterpret_cast<const uint32_t*>(
                                              static_cast<const uint8_t*>(rows) + (int64_t)idv[i] * d) + j + 8 * k)
                                        : 0u, 0u);
            else
                r[i][k] = ok ? __ldg(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(rows) +
                                                                    (int64_t)idv[i] * d) + j + 8 * k)
                             : make_uint2(0u, 0u);
        }
    float a[4];
    const float2 m23 = make_float2(8388608.f, 8388608.f);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k >= nch) break;  // warp-uniform
            float2 x01, x23;
            if (U8) {
                const uint32_t w = r[i][k].x;
                x01 = f2_sub(make_float2(__uint_as_float(prmt(w, 0x4B000000u, 0x7540u)),
                                         __uint_as_float(prmt(w, 0x4B000000u, 0x7541u))), m23);
                x23 = f2_sub(make_float2(__uint_as_float(prmt(w, 0x4B000000u, 0x7542u)),
                                         __uint_as_float(prmt(w, 0x4B000000u, 0x7543u))), m23);
            } else {
                x01 = make_float2(__uint_as_float(r[i][k].x << 16), __uint_as_float(r[i][k].x & 0xffff0000u));
                x23 = make_float2(__uint_as_float(r[i][k].y << 16), __uint_as_float(r[i][k].y & 0xffff0000u));
            }
            const float2 q01 = make_float2(qv[k].x, qv[k].y), q23 = make_float2(qv[k].z, qv[k].w);
            if (ip) {
                acc = f2_fma(q01, x01, acc);
                acc = f2_fma(q23, x23, acc);
            } else {
                const float2 e01 = f2_sub(q01, x01), e23 = f2_sub(q23, x23);
                acc = f2_fma(e01, e01, acc);
                acc = f2_fma(e23, e23, acc);
            }
        }
        a[i] = acc.x + acc.y;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 4;
        const float send = up ? a[i] : a[i + 2], keep = up ? a[i + 2] : a[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const float send = up ? a[0] : a[1], keep = up ? a[1] : a[0];
        a[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
    return a[0];
}

// U8: the band's rows are U8 (xu), else BF16 (xb).
template <bool U8>
__global__ void __launch_bounds__(RW_WARPS * 32) k_rerank_w(const float* __restrict__ Q, const float* __restrict__ X,
                                                            int d, int ip, const uint64_t* __restrict__ topr,
                                                            int Rmax, const int32_t* __restrict__ rerank_q, int Rfix,
                                                            int k, int64_t nq, int64_t* __restrict__ out_ids,
                                                            float* __restrict__ out_d,
                                                            const uint16_t* __restrict__ xb,
                                                            const uint8_t* __restrict__ xu,
                                                            const float2* __restrict__ xe) {
    // RW_WARPS x Rmax keys; with xb also RW_WARPS x Rmax bound pairs and RW_WARPS x (Rmax + 64) words
    extern __shared__ uint64_t wkeys[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * RW_WARPS + w;
    if (q >= nq) return;
    uint64_t* keys = wkeys + (size_t)w * Rmax;  // the candidates' keys, staged; then their FP32 keys
    const int R = rerank_of(rerank_q, Rfix, k, Rmax, q);
    const bool inl = lane * 4 < d;
    float4 qv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (inl) {  // the query matrix may be only 4-byte aligned
        const float* qp = Q + q * d + lane * 4;
        qv = make_float4(qp[0], qp[1], qp[2], qp[3]);
    }
    // the candidate keys in shared memory (one coalesced pass), so that a
    // step's row loads wait for a shared load, not for a global one
    {
        const uint64_t* cq = topr + q * Rmax;
        for (int c = lane; c < R; c += 32) keys[c] = cq[c];
        __syncwarp();
    }
    // row of the sum this lane holds after the exchange
    const int myrow = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    auto id_of = [&](int c) -> int32_t {
        const uint64_t kk = c < R ? keys[c] : KEY_NONE;
        return kk != KEY_NONE ? (int32_t)(kk & 0xffffffffu) : -1;
    };
    auto fp32_key = [&](uint64_t kk, float a0) -> uint64_t {
        return kk != KEY_NONE ? (((uint64_t)ordered_f32(ip ? -a0 : a0) << 32) | (kk & 0xffffffffull)) : KEY_NONE;
    };
    // the k smallest of arr[0..cnt) to the outputs: one warp sort when they
    // fit a warp, else k rounds of a warp minimum
    auto emit_best = [&](uint64_t* arr, int cnt) {
        uint64_t mine = KEY_NONE;  // lane r keeps the r-th smallest
        if (cnt <= 32) {
            mine = warp_sort_key(lane < cnt ? arr[lane] : KEY_NONE, lane);
        } else {
            for (int r = 0; r < k; ++r) {
                uint64_t m = KEY_NONE;
                int at = -1;
                for (int i = lane; i < cnt; i += 32) {
                    if (arr[i] < m) { m = arr[i]; at = i; }
                }
                uint64_t gk = m;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const uint64_t y = __shfl_xor_sync(0xffffffffu, gk, o);
                    gk = y < gk ? y : gk;
                }
                if (gk != KEY_NONE && m == gk) arr[at] = KEY_NONE;  // keys are unique: one lane matches
                __syncwarp();
                if (lane == r) mine = gk;
            }
        }
        if (lane < k) {
            if (mine == KEY_NONE) {
                out_ids[q * k + lane] = -1;
                out_d[q * k + lane] = ip ? -INFINITY : INFINITY;
            } else {
                out_ids[q * k + lane] = (int64_t)(mine & 0xffffffffu);
                const float dist = unordered_f32((uint32_t)(mine >> 32));
                out_d[q * k + lane] = ip ? -dist : dist;
            }
        }
    };
    if ((xb || xu) && R > k) {
        float2* band = reinterpret_cast<float2*>(wkeys + (size_t)RW_WARPS * Rmax) + (size_t)w * Rmax;
        uint32_t* sv = reinterpret_cast<uint32_t*>(wkeys + (size_t)2 * RW_WARPS * Rmax) + (size_t)w * (Rmax + 64);
        uint32_t* kv = sv + Rmax;  // the small selection's values
        const float g = 0x1p-20f, safe = 1.f + 0x1p-10f;
        float qn = 0.f;  // IP: an upper bound of |q|
        if (ip) {
            float t = fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, fmaf(qv.z, qv.z, qv.w * qv.w)));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            qn = sqrtf(t) * (1.f + 0x1p-18f);
        }
        // this lane's query chunks for the 8-lanes-per-row BF16 pass
        const int nch = (d + 31) >> 5;
        float4 qc[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int t0 = 4 * ((lane & 7) + 8 * h);
            qc[h] = t0 < d ? make_float4(Q[q * d + t0], Q[q * d + t0 + 1], Q[q * d + t0 + 2], Q[q * d + t0 + 3])
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int myrow16 = (lane >> 1) & 15;
        // the candidates' ids (-1: none) to 16 past R, in sv until the
        // survivors replace them: one shared load per row and step
        const int R16 = (R + 15) & ~15;
        for (int c = lane; c < R16; c += 32) sv[c] = (uint32_t)id_of(c);
        __syncwarp();
        for (int c0 = 0; c0 < R; c0 += 16) {
            int32_t idv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) idv[i] = (int32_t)sv[c0 + 4 * (lane >> 3) + i];
            // this lane's row bounds, loaded beside the rows
            const int c = c0 + myrow16;
            const int32_t id = (int32_t)sv[c];
            const float2 nr = id >= 0 ? __ldg(xe + id) : make_float2(0.f, 0.f);
            const float a0 = U8 ? rerank_rows16_band<true>(qc, xu, d, ip, nch, idv, lane)
                                : rerank_rows16_band<false>(qc, xb, d, ip, nch, idv, lane);
            if ((lane & 1) == 0 && c < R) {
                float lo = INFINITY, hi = INFINITY;
                if (id >= 0) {
                    const float n = nr.x, r = nr.y;
                    float e, dt;
                    if (ip) {
                        dt = -a0;
                        e = qn * (r + 2.01f * g * (n + r)) * safe;
                    } else {
                        dt = a0;
                        const float sq = sqrtf(fmaxf(dt, 0.f) * (1.f + 2.f * g)) * (1.f + 0x1p-20f);
                        e = (2.f * r * sq + r * r + g * (sq * sq + (sq + r) * (sq + r))) * safe;
                    }
                    lo = __fsub_rd(dt, e);
                    hi = __fadd_ru(dt, e);
                    if (!(lo <= hi)) {  // a NaN: no bound, the candidate is read in FP32
                        lo = -INFINITY;
                        hi = INFINITY;
                    }
                }
                band[c] = make_float2(lo, hi);
            }
        }
        __syncwarp();
        // U: the k-th smallest upper bound (+inf when the small selection
        // cannot tell: then every candidate is re-scored)
        float U = INFINITY;
        auto load_hi = [&](int c) -> uint32_t { return ordered_f32(band[c].y); };
        if (k <= 48 && warp_small_kvals(load_hi, R, k, kv) >= 0) U = unordered_f32(kv[k - 1]);
        // survivors: lower bound <= U
        const uint32_t below = (1u << lane) - 1u;
        int ns = 0;
        for (int c0 = 0; c0 < R; c0 += 32) {
            const int c = c0 + lane;
            const bool in = c < R && band[c].x <= U;
            const uint32_t m = __ballot_sync(0xffffffffu, in);
            if (in) sv[ns + __popc(m & below)] = (uint32_t)c;
            ns += __popc(m);
        }
        __syncwarp();
        // their FP32 keys, by survivor index, where the bounds were
        uint64_t* fk = reinterpret_cast<uint64_t*>(band);
        for (int s0 = 0; s0 < ns; s0 += 8) {
            int32_t idv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) idv[u] = s0 + u < ns ? id_of((int)sv[s0 + u]) : -1;
            const float a0 = rerank_rows8(qv, X, d, ip, inl, idv, lane);
            const int si = s0 + myrow;
            if ((lane & 3) == 0 && si < ns) fk[si] = fp32_key(keys[sv[si]], a0);
        }
        __syncwarp();
        emit_best(fk, ns);
    } else {
        for (int c0 = 0; c0 < R; c0 += 8) {
            int32_t idv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) idv[u] = id_of(c0 + u);
            const float a0 = rerank_rows8(qv, X, d, ip, inl, idv, lane);
            const int c = c0 + myrow;
            const uint64_t kk = c < R ? keys[c] : KEY_NONE;
            __syncwarp();  // this step's keys are read before they are replaced
            if ((lane & 3) == 0 && c < R) keys[c] = fp32_key(kk, a0);
        }
        __syncwarp();
        emit_best(keys, R);
    }
}

// Per row of X and of its low-precision copy (BF16 xb, or U8 xu): (an upper
// bound of |x|, an upper bound of |x~ - x|), each the sqrt of an FP64 sum of
// squares rounded up to FP32 (x~ - x is exact in FP64).  A row the copy holds
// exactly gets r = 0; a row with a non-finite coordinate gets r = +inf (every
// bound infinite).  A warp per row.
__global__ void k_band_rows(const float* __restrict__ X, const uint16_t* __restrict__ xb,
                            const uint8_t* __restrict__ xu, int64_t n, int d, float2* __restrict__ out) {
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    double s = 0.0, e = 0.0;
    for (int t = lane; t < d; t += 32) {
        const double v = X[r * d + t];
        const double w = xu ? (double)xu[r * d + t] : (double)__uint_as_float((uint32_t)xb[r * d + t] << 16);
        s += v * v;
        e += (v - w) * (v - w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    if (lane == 0) {
        float nb = __double2float_ru(sqrt(s) * (1.0 + 0x1p-40));
        float rb = e == 0.0 ? 0.f : __double2float_ru(sqrt(e) * (1.0 + 0x1p-40));
        if (!(nb < INFINITY) || !(rb < INFINITY)) nb = rb = INFINITY;
        out[r] = make_float2(nb, rb);
    }
}

// Clears *ok unless every element of X [m] is an integer in [0, 255] (a
// byte holds it exactly; -0 counts as 0).
__global__ void k_bytes_exact(const float* __restrict__ X, int64_t m, int32_t* __restrict__ ok) {
    bool all = true;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = X[i];
        all &= v >= 0.f && v <= 255.f && v == rintf(v);
    }
    if (!__all_sync(0xffffffffu, all) && (threadIdx.x & 31) == 0) atomicAnd(ok, 0);
}

__global__ void k_x_u8(const float* __restrict__ X, int64_t m, uint8_t* __restrict__ xu) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        xu[i] = (uint8_t)X[i];
}

// ------------------------------------------------------------------ precision variant
// Low-precision copies of X for the widened first re-rank: BF16 rows, or FP8
// e4m3 rows with one FP32 scale per row (x ~ fp8(x / s) * s, s = max|x| / 448).
__global__ void k_x_lowp(const float* __restrict__ X, int64_t n, int d, int prec, uint16_t* __restrict__ xb,
                         uint8_t* __restrict__ x8, float* __restrict__ sc) {
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float* x = X + r * d;
    if (prec == 1) {
        for (int t = lane; t < d; t += 32) xb[r * d + t] = __bfloat16_as_ushort(__float2bfloat16_rn(x[t]));
        return;
    }
    float mx = 0.f;
    for (int t = lane; t < d; t += 32) mx = fmaxf(mx, fabsf(x[t]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float s = mx > 0.f ? mx / 448.f : 1.f;
    if (lane == 0) sc[r] = s;
    for (int t = lane; t < d; t += 32)
        x8[r * d + t] = (uint8_t)__nv_cvt_float_to_fp8(x[t] / s, __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ float lowp_elem(int prec, const uint16_t* xb, const uint8_t* x8, int64_t off) {
    if (prec == 1) return __bfloat162float(__ushort_as_bfloat16(xb[off]));
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)x8[off], __NV_E4M3);
    return __half2float(__half(h));
}

// Distance of query row qs (shared) to row id in the given precision (0 FP32,
// 1 BF16, 2 FP8 with row scale); one warp, result in every lane.
__device__ __forceinline__ float lowp_dist(int prec, const float* __restrict__ qs, const float* __restrict__ X,
                                           const uint16_t* __restrict__ xb, const uint8_t* __restrict__ x8,
                                           const float* __restrict__ sc, int32_t id, int d, int ip, int lane) {
    float acc = 0.f;
    const float s = prec == 2 ? sc[id] : 1.f;
    for (int t = lane; t < d; t += 32) {
        const float xv = prec == 0 ? __ldg(X + (int64_t)id * d + t) : lowp_elem(prec, xb, x8, (int64_t)id * d + t) * s;
        if (ip) acc = fmaf(qs[t], xv, acc);
        else { const float e = qs[t] - xv; acc = fmaf(e, e, acc); }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return ip ? -acc : acc;
}

// Widened first re-rank: the R_w candidates (topr) by low-precision
// distance, the best Rf of them (by (distance, id)) written as keys to out.
__global__ void __launch_bounds__(256) k_rerank_lowp(const float* __restrict__ Q, int d, int ip, int prec,
                                                     const uint16_t* __restrict__ xb, const uint8_t* __restrict__ x8,
                                                     const float* __restrict__ sc, const uint64_t* __restrict__ topr,
                                                     int Rmax, const int32_t* __restrict__ rerank_q, int Rfix,
                                                     int Rmin, int Rf, uint64_t* __restrict__ out) {
    extern __shared__ uint64_t keys[];
    __shared__ __align__(16) float qs[KSC_MAX_DIM];
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int R = rerank_of(rerank_q, Rfix, Rmin, Rmax, q);
    for (int t = threadIdx.x; t < d; t += blockDim.x) qs[t] = Q[q * d + t];
    __syncthreads();
    const uint64_t* cq = topr + q * Rmax;
    for (int c = w; c < R; c += nw) {
        const uint64_t kk = cq[c];
        uint64_t o = KEY_NONE;
        if (kk != KEY_NONE) {
            const int32_t id = (int32_t)(kk & 0xffffffffu);
            o = ((uint64_t)ordered_f32(lowp_dist(prec, qs, nullptr, xb, x8, sc, id, d, ip, lane)) << 32) | (uint32_t)id;
        }
        if (lane == 0) keys[c] = o;
    }
    const int S = pow2_ceil(R < 2 ? 2 : R);
    for (int i = R + threadIdx.x; i < S; i += blockDim.x) keys[i] = KEY_NONE;
    __syncthreads();
    block_bitonic_sort(keys, S);
    for (int i = threadIdx.x; i < Rf; i += blockDim.x) out[q * Rf + i] = i < R ? keys[i] : KEY_NONE;
}

// Diagnostic: distances of given (query, id) pairs in a precision.
__global__ void k_pair_dist(const float* __restrict__ Q, int64_t nq, int d, int ip, int prec,
                            const float* __restrict__ X, const uint16_t* __restrict__ xb,
                            const uint8_t* __restrict__ x8, const float* __restrict__ sc,
                            const int64_t* __restrict__ ids, int c, float* __restrict__ out) {
    __shared__ __align__(16) float qs[KSC_MAX_DIM];
    const int64_t q = blockIdx.x;
    for (int t = threadIdx.x; t < d; t += blockDim.x) qs[t] = Q[q * d + t];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = w; i < c; i += nw) {
        const int64_t id = ids[q * c + i];
        const float v = id >= 0 ? lowp_dist(prec, qs, X, xb, x8, sc, (int32_t)id, d, ip, lane) : NAN;
        if (lane == 0) out[q * c + i] = ip ? -v : v;
    }
}

// Candidate export: each query's R selected keys, ascending (the select
// leaves them unordered).  One CTA per query.
__global__ void __launch_bounds__(256) k_copy_cands(const uint64_t* __restrict__ topr, int Rmax,
                                                    uint64_t* __restrict__ out) {
    extern __shared__ uint64_t cs[];
    const int64_t q = blockIdx.x;
    const int S = pow2_ceil(Rmax < 2 ? 2 : Rmax);
    for (int i = threadIdx.x; i < S; i += blockDim.x) cs[i] = i < Rmax ? topr[q * Rmax + i] : KEY_NONE;
    __syncthreads();
    block_bitonic_sort(cs, S);
    for (int i = threadIdx.x; i < Rmax; i += blockDim.x) out[q * Rmax + i] = cs[i];
}

// ------------------------------------------------------------------ host pipeline
// Stage boundary i (0 = start of stage 0, KSC_NUM_STAGES = end of the last).
static void mark(ksc_index* ix, int i, cudaStream_t st) {
    if (!ix->prof) return;
    cudaEventRecord(ix->ev[i], st);
    ix->ev_used[i] = true;
}

static unsigned blocks_for(int64_t work, int threads) { return (unsigned)((work + threads - 1) / threads); }

struct Plan {
    int64_t nq;
    int k, Pmax, Rmax, Pfix, Rfix;
    const int32_t* nprobe_q;
    const int32_t* rerank_q;
    int G, TB, TBa, cap;  // TB: tile blocks of the filtered scan, TBa: of the unfiltered first part
    int rank_mode;  // RankMode of the list scores
    bool hybrid;
    int n_near, efs, tau;
    int prec, Rf;  // precision variant: first re-rank of R (= Rmax) in prec, then FP32 of the best Rf
    bool band;     // exact re-rank with the band of U8 / BF16 rows (k_rerank_w)
    int Pq_max;    // bound on the per-query nprobe (<= Pmax)
    bool tc;       // scan on the tensor cores (k_scan_tc)
    int nt;        // its queries per item
};

static int choose_G(const ksc_index* ix, int64_t nq, int Pmax, int want) {
    if (want == 4 && ix->M <= 128) return 4;
    if (want == 8 || want == 16 || want == 32) {
        int S = (ix->M + want - 1) / want;
        if (S <= 16) return want;
    }
    // 8 lanes per query (4 query slots per warp) up to 128 subspaces: when
    // fewer queries than slots probe a list, the item's slots split its
    // blocks instead, so every lane stays busy at any batch size, and the
    // per-block reduction runs over 8 lanes only
    (void)nq;
    (void)Pmax;
    if (ix->M <= 128) return 8;
    if (ix->M <= 256) return 16;
    return 32;
}

template <int G, int SMAX>
static int launch_scan(const ScanArgs& A, const ScanOut& O, const int64_t* pair_off, const int64_t* item_off,
                       const uint32_t* pairs, int L, int TB, int32_t* status, cudaStream_t st) {
    const size_t smem = (size_t)SCAN_WARPS * 2 * scan_chunk_bytes<G>() +
                        (scan_shared_sel<G>() ? (size_t)SCAN_WARPS * A.M * 64 : 0);
    // M = G SMAX: every lane has SMAX subspaces, no per-subspace guards
    const bool full = A.M == G * SMAX;
    auto kern = O.thr ? (full ? k_scan<G, SMAX, false, true> : k_scan<G, SMAX, false, false>)
                      : (full ? k_scan<G, SMAX, true, true> : k_scan<G, SMAX, true, false>);
    KSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    KSC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SCAN_WARPS * 32, smem));
    const int grid = num_sms() * (per_sm > 0 ? per_sm : 1);
    kern<<<grid, SCAN_WARPS * 32, smem, st>>>(A, O, pair_off, item_off, pairs, L, TB, status);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

template <int MAXM>
static int launch_scan4(const ScanArgs& A, const ScanOut& O, const int64_t* pair_off, const int64_t* item_off,
                        const uint32_t* pairs, int L, int TB, int32_t* status, cudaStream_t st) {
    const size_t smem = (size_t)S4_WARPS * s4_warp_bytes<MAXM>();
    KSC_CUDA(cudaFuncSetAttribute(k_scan4<MAXM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    KSC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan4<MAXM>, S4_WARPS * 32, smem));
    const int grid = num_sms() * (per_sm > 0 ? per_sm : 1);
    k_scan4<MAXM><<<grid, S4_WARPS * 32, smem, st>>>(A, O, pair_off, item_off, pairs, L, TB, status);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

template <int G>
static int dispatch_scan(int S, const ScanArgs& A, const ScanOut& O, const int64_t* pair_off,
                         const int64_t* item_off, const uint32_t* pairs, int L, int TB, int32_t* status,
                         cudaStream_t st) {
    if (S <= 2) return launch_scan<G, 2>(A, O, pair_off, item_off, pairs, L, TB, status, st);
    if (S <= 4) return launch_scan<G, 4>(A, O, pair_off, item_off, pairs, L, TB, status, st);
    if constexpr (G == 8)
        if (S == 6) return launch_scan<G, 6>(A, O, pair_off, item_off, pairs, L, TB, status, st);  // M 48
    if (S <= 8) return launch_scan<G, 8>(A, O, pair_off, item_off, pairs, L, TB, status, st);
    if (S <= 16) return launch_scan<G, 16>(A, O, pair_off, item_off, pairs, L, TB, status, st);
    set_error("M too large for %d lanes per query", G);
    return KSC_EINVAL;
}

// Operand type of the list scores (a1): 16-bit tensor cores, FP32 CUDA
// cores, or FP8 tensor cores.
enum RankMode { RANK_TC16 = 0, RANK_FP32 = 1, RANK_FP8 = 2 };

// List scores [nq x L] on the 16-bit or FP8 tensor cores or the FP32 CUDA
// cores, with the per-query bound err [nq] on their distance from the exact
// scores.
static int list_scores(ksc_index* ix, const float* Q, int64_t nq, int mode, float* scores, float** err,
                       cudaStream_t st) {
    KSC_TRY(ensure(ix->ws_err, sizeof(float) * nq, st));
    *err = (float*)ix->ws_err.p;
    if (mode != RANK_FP32 && tc_rank_supported(ix))
        return mode == RANK_FP8 ? rank_scores_tc8(ix, Q, nq, scores, *err, st)
                                : rank_scores_tc(ix, Q, nq, scores, *err, st);
    dim3 grid(blocks_for(ix->L, SC_T), blocks_for(nq, SC_T));
    k_list_scores<<<grid, 256, 0, st>>>(Q, nq, ix->d, ix->c_rank, ix->c_rank_sq, ix->L, ix->spherical, scores);
    ix->launches++;
    KSC_LAUNCH_CHECK();
    return score_err(ix, Q, nq, false, *err, st);
}

// The Pmax best lists of every query (exact ranking); feat (optional, L >=
// FEAT_K) receives each query's FEAT_K smallest given list distances.
// The warp kernel ranks a batch when its lists fit a warp's share of shared
// memory and the batch fills the GPU.
static bool rank_by_warp(const ksc_index* ix, int64_t nq, int Pmax) {
    return ix->L <= RSW_MAX_L && Pmax <= 4 * RSW_CAND / 8 && warp_per_query(nq);
}

// The P best lists of every query from the given approximate scores (an
// error bound per query in err), exactly re-scored; feat: the predictor's
// distances as well.
static int select_lists(ksc_index* ix, const float* scores, const float* err, const float* Q, int64_t nq,
                        const int32_t* nprobe_q, int Pfix, int Pmax, int32_t* probes, float* score_out,
                        cudaStream_t st, float* feat);

static int rank_lists(ksc_index* ix, const float* Q, int64_t nq, const int32_t* nprobe_q, int Pfix, int Pmax,
                      int32_t* probes, float* score_out, int mode, cudaStream_t st, float* feat = nullptr) {
    KSC_TRY(ensure(ix->ws_scores, sizeof(float) * nq * ix->L, st));
    float* scores = (float*)ix->ws_scores.p;
    float* err = nullptr;
    KSC_TRY(list_scores(ix, Q, nq, mode, scores, &err, st));
    return select_lists(ix, scores, err, Q, nq, nprobe_q, Pfix, Pmax, probes, score_out, st, feat);
}

static int select_lists(ksc_index* ix, const float* scores, const float* err, const float* Q, int64_t nq,
                        const int32_t* nprobe_q, int Pfix, int Pmax, int32_t* probes, float* score_out,
                        cudaStream_t st, float* feat) {
    // re-score buffer of the CTA kernel: 4 Pmax lists (a power of two, at least 1024, at most RS_CAP)
    const int rs_cap = std::min(RS_CAP, std::max(1024, pow2_ceil(4 * Pmax)));
    const size_t smem = rs_cap * sizeof(uint64_t) + (ix->L <= RS_SMEM_L ? sizeof(float) * ix->L : 0);
    KSC_CUDA(cudaFuncSetAttribute(k_rank_select<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    KSC_CUDA(cudaFuncSetAttribute(k_rank_select<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (rank_by_warp(ix, nq, Pmax)) {
        // a warp per query; queries with too many lists inside the bound go to the CTA kernel
        KSC_TRY(ensure(ix->ws_redo, sizeof(int32_t) * (nq + 1), st));
        int32_t* redo = (int32_t*)ix->ws_redo.p;
        KSC_CUDA(cudaMemsetAsync(redo, 0, sizeof(int32_t), st));
        const size_t wsm = sizeof(uint64_t) * RSW_WARPS * RSW_CAND + sizeof(float) * RSW_WARPS * ix->L;
        KSC_CUDA(cudaFuncSetAttribute(k_rank_select_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm));
        k_rank_select_w<<<(unsigned)((nq + RSW_WARPS - 1) / RSW_WARPS), RSW_WARPS * 32, wsm, st>>>(
            scores, err, Q, ix->c_rank, nq, ix->d, ix->L, ix->spherical, nprobe_q, Pfix, Pmax, probes, score_out,
            redo, feat);
        feat = nullptr;  // written
        KSC_LAUNCH_CHECK();
        k_rank_select<256><<<num_sms() * 2, 256, smem, st>>>(scores, err, Q, ix->c_rank, nq, ix->d, ix->L, ix->spherical,
                                                        nprobe_q, Pfix, Pmax, rs_cap, probes, score_out, redo);
        ix->launches += 2;
    } else {
        // a CTA per query; 1024 threads when the batch is too small to fill the GPU
        if (nq < 2 * (int64_t)num_sms())
            k_rank_select<1024><<<(unsigned)nq, 1024, smem, st>>>(scores, err, Q, ix->c_rank, nq, ix->d, ix->L,
                                                                  ix->spherical, nprobe_q, Pfix, Pmax, rs_cap, probes,
                                                                  score_out, nullptr);
        else
            k_rank_select<256><<<(unsigned)nq, 256, smem, st>>>(scores, err, Q, ix->c_rank, nq, ix->d, ix->L,
                                                                ix->spherical, nprobe_q, Pfix, Pmax, rs_cap, probes,
                                                                score_out, nullptr);
        ix->launches++;
    }
    KSC_LAUNCH_CHECK();
    if (feat) {
        k_feat_scores<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(scores, Q, ix->d, ix->spherical, nq, ix->L, feat);
        KSC_LAUNCH_CHECK();
        ix->launches++;
    }
    return KSC_OK;
}

static int launch_luts(const LutArgs& A, uint32_t* rb, uint8_t* lut, int32_t* bias, float* scale, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)A.M * cb_ld(A.dsub);
    const int64_t warps = (A.nq * A.Pmax + LUT_WARPS - 1) / LUT_WARPS;  // a warp per item
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(warps, (int64_t)num_sms() * 8));
    if (lut_ds2(A)) {
        KSC_CUDA(cudaFuncSetAttribute(k_lut_range<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        KSC_CUDA(cudaFuncSetAttribute(k_lut_quant<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_lut_range<2><<<grid, LUT_WARPS * 32, smem, st>>>(A, rb);
        KSC_LAUNCH_CHECK();
        k_lut_quant<2><<<grid, LUT_WARPS * 32, smem, st>>>(A, rb, lut, bias, scale);
    } else {
        KSC_CUDA(cudaFuncSetAttribute(k_lut_range<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        KSC_CUDA(cudaFuncSetAttribute(k_lut_quant<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_lut_range<0><<<grid, LUT_WARPS * 32, smem, st>>>(A, rb);
        KSC_LAUNCH_CHECK();
        k_lut_quant<0><<<grid, LUT_WARPS * 32, smem, st>>>(A, rb, lut, bias, scale);
    }
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

static int compute_luts(ksc_index* ix, const float* Q, int64_t nq, const int32_t* probes, const int32_t* nprobe_q,
                        int Pfix, int Pmax, uint8_t* lut, int32_t* bias, float* scale, cudaStream_t st) {
    KSC_TRY(ensure(ix->ws_range, sizeof(uint32_t) * nq, st));
    uint32_t* rb = (uint32_t*)ix->ws_range.p;
    KSC_CUDA(cudaMemsetAsync(rb, 0, sizeof(uint32_t) * nq, st));
    LutArgs A{Q, nq, ix->d, ix->M, ix->dsub, ix->metric == KSC_IP, Pmax, probes, nprobe_q, Pfix, ix->c_mean,
              ix->codebook, ix->L};
    KSC_TRY(launch_luts(A, rb, lut, bias, scale, st));
    ix->launches += 2;
    return KSC_OK;
}

// BF16 / FP8 copies of the re-rank vectors, made on first use.
static int ensure_lowp(ksc_index* ix, int prec, cudaStream_t st) {
    const int dr = rr_d(ix);
    if (prec == 1 && !ix->X_bf16) {
        KSC_CUDA(cudaMalloc(&ix->X_bf16, sizeof(uint16_t) * ix->n * dr));
        k_x_lowp<<<(unsigned)((ix->n + 7) / 8), 256, 0, st>>>(rr_X(ix), ix->n, dr, 1, (uint16_t*)ix->X_bf16, nullptr,
                                                              nullptr);
        KSC_LAUNCH_CHECK();
    }
    if (prec == 2 && !ix->X_fp8) {
        KSC_CUDA(cudaMalloc(&ix->X_fp8, (size_t)ix->n * dr));
        KSC_CUDA(cudaMalloc(&ix->X_scale, sizeof(float) * ix->n));
        k_x_lowp<<<(unsigned)((ix->n + 7) / 8), 256, 0, st>>>(rr_X(ix), ix->n, dr, 2, nullptr, (uint8_t*)ix->X_fp8,
                                                              ix->X_scale);
        KSC_LAUNCH_CHECK();
    }
    return KSC_OK;
}

// The band of the exact re-rank, made on first use: U8 copies of the rows
// when every coordinate is an integer in [0, 255] (checked once; exact, a
// quarter of the FP32 bytes), else BF16 copies; and the rows' bounds (norm,
// rounding error).
static int ensure_band(ksc_index* ix, cudaStream_t st) {
    const int64_t m = ix->n * (int64_t)rr_d(ix);
    if (ix->x_u8_state == 0) {
        KSC_TRY(ensure(ix->ws_flag, sizeof(int32_t), st));
        int32_t* ok = (int32_t*)ix->ws_flag.p;
        const int32_t one = 1;
        KSC_CUDA(cudaMemcpyAsync(ok, &one, sizeof(int32_t), cudaMemcpyHostToDevice, st));
        k_bytes_exact<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 8 * (int64_t)num_sms())),
                        256, 0, st>>>(rr_X(ix), m, ok);
        KSC_LAUNCH_CHECK();
        int32_t h = 0;
        KSC_CUDA(cudaMemcpyAsync(&h, ok, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        KSC_CUDA(cudaStreamSynchronize(st));
        if (h && m > 0 && !ix->X_u8) {
            KSC_CUDA(cudaMalloc(&ix->X_u8, (size_t)m));
            k_x_u8<<<(unsigned)std::min<int64_t>((m + 255) / 256, 8 * (int64_t)num_sms()), 256, 0, st>>>(
                rr_X(ix), m, (uint8_t*)ix->X_u8);
            KSC_LAUNCH_CHECK();
        }
        ix->x_u8_state = (h && m > 0) ? 1 : -1;  // only once the copy exists
    }
    const bool u8 = ix->x_u8_state == 1;
    if (!u8) KSC_TRY(ensure_lowp(ix, 1, st));
    if (!ix->X_band) {
        KSC_CUDA(cudaMalloc(&ix->X_band, sizeof(float2) * ix->n));
        k_band_rows<<<(unsigned)((ix->n + 7) / 8), 256, 0, st>>>(
            rr_X(ix), u8 ? nullptr : (const uint16_t*)ix->X_bf16, u8 ? (const uint8_t*)ix->X_u8 : nullptr, ix->n,
            rr_d(ix), ix->X_band);
        KSC_LAUNCH_CHECK();
    }
    return KSC_OK;
}

// Cluster-major work list of the (query, rank) pairs of one part of the probe
// ranks (the unfiltered first part or the rest).
struct WorkList {
    int64_t* pair_off;  // [L + 1]
    int64_t* item_off;  // [L + 1]
    int32_t* cnt;       // [L]
    int32_t* fill;      // [L]
    uint32_t* pairs;    // [<= nq * Pmax]
    int TB;             // blocks per item tile
};

static int run_scan(const Plan& pl, int M, const ScanArgs& A, const ScanOut& O, const WorkList& w, int L,
                    int32_t* status, cudaStream_t st, unsigned long long* next_item, bool tc) {
    if (tc) return launch_scan_tc(A, O, w.pair_off, w.item_off, w.pairs, L, w.TB, pl.nt, next_item, status, st);
    const int S = (M + pl.G - 1) / pl.G;
    if (pl.G == 4) {
        if (M <= 64) return launch_scan4<64>(A, O, w.pair_off, w.item_off, w.pairs, L, w.TB, status, st);
        if (M <= 128) return launch_scan4<128>(A, O, w.pair_off, w.item_off, w.pairs, L, w.TB, status, st);
        set_error("M too large for 4 lanes per query");
        return KSC_EINVAL;
    }
    if (pl.G == 8) return dispatch_scan<8>(S, A, O, w.pair_off, w.item_off, w.pairs, L, w.TB, status, st);
    if (pl.G == 16) return dispatch_scan<16>(S, A, O, w.pair_off, w.item_off, w.pairs, L, w.TB, status, st);
    return dispatch_scan<32>(S, A, O, w.pair_off, w.item_off, w.pairs, L, w.TB, status, st);
}

// a2 .. a6 for given probe lists.  Stages: 1 work lists, 2 LUTs, 3 scan of
// the nearest list(s) + threshold, 4 scan of the other lists, 5 select,
// 6 rerank.
// Queries in the index's working dimensions: with component filtration
// (Sec. 4.3, Alg. 2 FilterComponents) the kept dimensions of Q, gathered into
// a workspace buffer (zeros in the padding); otherwise Q itself.
static int work_queries(ksc_index* ix, const float* Q, int64_t nq, cudaStream_t st, const float** Qw) {
    *Qw = Q;
    if (!ix->dims || nq == 0) return KSC_OK;
    KSC_TRY(ensure(ix->ws_qf, sizeof(float) * nq * ix->d, st));
    KSC_TRY(gather_dims(Q, nq, ix->d_rr, ix->dims, ix->d, (float*)ix->ws_qf.p, st));
    ix->launches++;
    *Qw = (const float*)ix->ws_qf.p;
    return KSC_OK;
}

// Q: the queries in the index's (working) dimensions; Qr: the same queries
// with all their dimensions for the re-rank (null: Q; they differ only under
// component filtration).
static int search_from_probes(ksc_index* ix, const float* Q, const Plan& pl, const int32_t* probes,
                              int64_t* ids, float* dists, uint64_t* cand_out, int32_t* ncand_out, cudaStream_t st,
                              const float* Qr = nullptr) {
    const int64_t nq = pl.nq;
    const int M = ix->M, L = ix->L;
    // queries per work item: the unfiltered first part always runs the
    // byte-permute scan (few queries share a list there: too few columns for
    // the tensor cores); the rest the chosen scan
    const int QGa = 32 / pl.G;
    const int QG = pl.tc ? pl.nt : QGa;
    // hybrid: the n_near nearest lists are the fully scanned ones (Sec. 4.4);
    // plain: a per-query split (k_count_parts)
    const int rA = std::min(pl.hybrid ? pl.n_near : 1, pl.Pmax);
    KSC_TRY(ensure(ix->ws_lut, (size_t)nq * pl.Pmax * M * PQ_K, st));
    KSC_TRY(ensure(ix->ws_bias, sizeof(int32_t) * nq * pl.Pmax, st));
    KSC_TRY(ensure(ix->ws_scale, sizeof(float) * nq, st));
    KSC_TRY(ensure(ix->ws_thr, sizeof(uint64_t) * nq, st));
    KSC_TRY(ensure(ix->ws_cnt, sizeof(int32_t) * nq, st));
    KSC_TRY(ensure(ix->ws_cand, sizeof(uint64_t) * nq * pl.cap, st));
    KSC_TRY(ensure(ix->ws_topr, sizeof(uint64_t) * nq * pl.Rmax, st));
    const size_t wl_head = sizeof(int64_t) * 2 * (L + 1) + sizeof(int32_t) * 2 * L;  // per work list
    KSC_TRY(ensure(ix->ws_items, 2 * wl_head + sizeof(uint32_t) * nq * (2 * pl.Pmax + 1) + 320, st));
    uint8_t* lut = (uint8_t*)ix->ws_lut.p;
    int32_t* bias = (int32_t*)ix->ws_bias.p;
    float* scale = (float*)ix->ws_scale.p;
    uint64_t* thr = (uint64_t*)ix->ws_thr.p;
    int32_t* cnt = (int32_t*)ix->ws_cnt.p;
    uint64_t* cand = (uint64_t*)ix->ws_cand.p;
    uint64_t* topr = (uint64_t*)ix->ws_topr.p;
    // both work lists side by side: pair_off [2][L+1], item_off [2][L+1],
    // cnt [2][L], fill [2][L], then the pairs
    WorkList wa, wb;
    {
        int64_t* po = (int64_t*)ix->ws_items.p;
        int64_t* io = po + 2 * (L + 1);
        int32_t* cn = (int32_t*)(io + 2 * (L + 1));
        int32_t* fl = cn + 2 * L;
        wa.pair_off = po;
        wb.pair_off = po + (L + 1);
        wa.item_off = io;
        wb.item_off = io + (L + 1);
        wa.cnt = cn;
        wb.cnt = cn + L;
        wa.fill = fl;
        wb.fill = fl + L;
        wa.pairs = (uint32_t*)(fl + 2 * L);
        wb.pairs = wa.pairs + nq * pl.Pmax;
    }
    int32_t* split = pl.hybrid ? nullptr : (int32_t*)(wb.pairs + nq * pl.Pmax);
    // item counters of the two tensor-core scans, after the split array
    unsigned long long* tc_next = reinterpret_cast<unsigned long long*>(
        (reinterpret_cast<uintptr_t>(wb.pairs + nq * pl.Pmax + nq) + 15) & ~uintptr_t(15));
    ScanArgs A{M, pl.Pmax, nq, probes, pl.nprobe_q, pl.Pfix, pl.rerank_q, pl.Rfix, pl.k, lut, bias,
               ix->list_boff, ix->list_n, ix->blk_codes, ix->blk_ids, ix->L};
    // 1. work lists: the nearest list of every query, and the rest
    mark(ix, 1, st);
    KSC_CUDA(cudaMemsetAsync(wa.cnt, 0, sizeof(int32_t) * 2 * L, st));
    if (pl.tc) KSC_CUDA(cudaMemsetAsync(tc_next, 0, 2 * sizeof(unsigned long long), st));
    k_count_parts<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(A, pl.Rmax, pl.cap, rA, split, wa.cnt, wb.cnt, cnt);
    wa.TB = pl.TBa;
    wb.TB = pl.TB;
    k_scan_lists<<<2, 1024, 0, st>>>(wa.cnt, ix->list_n, L, QGa, QG, wa.TB, wb.TB, wa.pair_off, wa.item_off,
                                     wa.fill);
    k_fill_parts<<<blocks_for(nq * pl.Pmax, 256), 256, 0, st>>>(A, rA, split, wa.pair_off, wa.fill, wa.pairs,
                                                                wb.pair_off, wb.fill, wb.pairs);
    KSC_LAUNCH_CHECK();
    ix->launches += 3;
    // 2. quantised LUTs of every probed (query, list)
    mark(ix, 2, st);
    {
        KSC_TRY(ensure(ix->ws_range, sizeof(uint32_t) * nq, st));
        uint32_t* rb = (uint32_t*)ix->ws_range.p;
        KSC_CUDA(cudaMemsetAsync(rb, 0, sizeof(uint32_t) * nq, st));
        LutArgs LA{Q, nq, ix->d, M, ix->dsub, ix->metric == KSC_IP, pl.Pmax, probes, pl.nprobe_q, pl.Pfix,
                   ix->c_mean, ix->codebook, ix->L, wa.pairs, wa.pair_off + L, wb.pairs, wb.pair_off + L};
        // tables stored for up to Pb probes per query (per-query nprobe: 8, the
        // rest of a larger query recomputed), so that more CTAs fit per SM
        const int Pb = pl.nprobe_q ? std::min(pl.Pq_max, 8) : pl.Pq_max;
        const size_t fsm = lut_fused_smem(M, ix->dsub, ix->d, Pb, pl.Pq_max);
        // one CTA per query at a time: worth it once every SM has queries to take
        if (fsm <= 160 * 1024 && nq >= 2 * (int64_t)num_sms()) {
            const bool ds2 = lut_ds2(LA);
            auto kf = ds2 ? k_lut_fused<2> : k_lut_fused<0>;
            KSC_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
            int per_sm = 0;
            KSC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, 256, fsm));
            const int64_t grid = std::min<int64_t>(nq, (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1));
            kf<<<(unsigned)grid, 256, fsm, st>>>(LA, Pb, pl.Pq_max, lut, bias, scale);
            KSC_LAUNCH_CHECK();
            ix->launches++;
        } else {
            KSC_TRY(launch_luts(LA, rb, lut, bias, scale, st));
            ix->launches += 2;
        }
    }
    // 3. scan of the nearest lists with no filter, then the threshold
    mark(ix, 3, st);
    KSC_TRY(run_scan(pl, M, A, ScanOut{nullptr, cnt, cand, pl.cap}, wa, L, ix->status, st, tc_next, false));
    // expected keys per query of the unfiltered scan: max(4 R, N / 16), N from
    // the mean list length; a warp per query up to SW_MAX_KEYS, else a CTA
    if (std::max(4.0 * pl.Rmax, (double)pl.Pmax * ix->n / L / 16.0) <= SW_MAX_KEYS && warp_per_query(nq))
        k_threshold<<<(unsigned)((nq + SW_WARPS - 1) / SW_WARPS), SW_WARPS * 32, 0, st>>>(A, pl.Rmax, cnt, cand,
                                                                                           pl.cap, topr, thr);
    else if (nq < 2 * (int64_t)num_sms())  // few queries: more threads per query
        k_threshold_cta<1024><<<(unsigned)nq, 1024, 0, st>>>(A, pl.Rmax, cnt, cand, pl.cap, topr, thr);
    else
        k_threshold_cta<256><<<(unsigned)nq, 256, 0, st>>>(A, pl.Rmax, cnt, cand, pl.cap, topr, thr);
    KSC_LAUNCH_CHECK();
    ix->launches += 2;
    // 4. scan of the other lists, keeping keys at or below the threshold;
    //    hybrid: graph search of every other list first, full scans only of
    //    the lists it marks (Sec. 4.4)
    mark(ix, 4, st);
    if (pl.hybrid) {
        KSC_TRY(ensure(ix->ws_full, sizeof(uint32_t) * nq * pl.Pmax + 64, st));
        int64_t* nfull = (int64_t*)ix->ws_full.p;
        uint32_t* full = (uint32_t*)(nfull + 2);
        KSC_CUDA(cudaMemsetAsync(nfull, 0, sizeof(int64_t), st));
        const int vwords = (((ix->max_list + 31) / 32) + 1) & ~1;  // even: keeps every warp's keys 8-byte aligned
        GraphArgs Gr{ix->nbr_pos, ix->nbr_codes, ix->entry_pos, pl.efs, pl.tau, vwords, full, nfull};
        const size_t smem = (size_t)GS_WARPS * ((size_t)GS_N * 16 + (size_t)vwords * 4);
        KSC_CHECK_ARG(smem <= 200 * 1024, "lists too large for the hybrid search (%d members)", ix->max_list);
        const int Sg = (M + 31) / 32;
        const int grid = num_sms() * 8;
        const ScanOut Og{thr, cnt, cand, pl.cap};
#define KSC_GS(SM)                                                                                        \
    do {                                                                                                  \
        KSC_CUDA(cudaFuncSetAttribute(k_graph_search<SM>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                      (int)smem));                                                        \
        k_graph_search<SM><<<grid, GS_WARPS * 32, smem, st>>>(A, Og, Gr, wb.pairs, wb.pair_off + L);      \
    } while (0)
        if (Sg <= 2) KSC_GS(2);
        else if (Sg <= 4) KSC_GS(4);
        else KSC_GS(8);
#undef KSC_GS
        KSC_LAUNCH_CHECK();
        // work list of the marked lists, then their scan
        KSC_CUDA(cudaMemsetAsync(wb.cnt, 0, sizeof(int32_t) * L, st));
        const int64_t nmax = nq * pl.Pmax;
        k_count_from<<<blocks_for(nmax, 256), 256, 0, st>>>(full, nfull, probes, wb.cnt);
        k_scan_lists<<<1, 1024, 0, st>>>(wb.cnt, ix->list_n, L, QG, QG, wb.TB, wb.TB, wb.pair_off, wb.item_off,
                                         wb.fill);
        k_fill_from<<<blocks_for(nmax, 256), 256, 0, st>>>(full, nfull, probes, wb.pair_off, wb.fill, wb.pairs);
        KSC_LAUNCH_CHECK();
        ix->launches += 4;
    }
    KSC_TRY(run_scan(pl, M, A, ScanOut{thr, cnt, cand, pl.cap}, wb, L, ix->status, st, tc_next + 1, pl.tc));
    ix->launches++;
    // 5. the R best keys per query
    mark(ix, 5, st);
    {
        KSC_TRY(ensure(ix->ws_redo, sizeof(int32_t) * (nq + 1), st));
        int32_t* redo = (int32_t*)ix->ws_redo.p;
        KSC_CUDA(cudaMemsetAsync(redo, 0, sizeof(int32_t), st));
        // candidates per query: the R kept by the threshold plus a few R more
        if (4 * pl.Rmax <= SW_MAX_KEYS && warp_per_query(nq))
            k_select<<<(unsigned)((nq + SW_WARPS - 1) / SW_WARPS), SW_WARPS * 32, 0, st>>>(
                A, pl.Rmax, cnt, cand, pl.cap, topr, ncand_out, ix->status, ix->stats, redo);
        else if (nq < 2 * (int64_t)num_sms())  // few queries: more threads per query
            k_select_cta<1024><<<(unsigned)nq, 1024, 0, st>>>(A, pl.Rmax, cnt, cand, pl.cap, topr, ncand_out,
                                                               ix->status, ix->stats, redo);
        else
            k_select_cta<256><<<(unsigned)nq, 256, 0, st>>>(A, pl.Rmax, cnt, cand, pl.cap, topr, ncand_out,
                                                             ix->status, ix->stats, redo);
        KSC_LAUNCH_CHECK();
        // overflowed queries (usually none): radix select over recomputed keys,
        // the R best plus their sort in a buffer of sel_cap keys
        const int sel_cap = sel_keys(pl.Rmax);
        const size_t smem = sel_cap * sizeof(uint64_t);
        KSC_CUDA(cudaFuncSetAttribute(k_select_redo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_select_redo<<<num_sms() * 2, 256, smem, st>>>(A, pl.Rmax, sel_cap, topr, ncand_out, redo);
        KSC_LAUNCH_CHECK();
        ix->launches += 2;
    }
    if (cand_out) {
        const size_t csm = sizeof(uint64_t) * pow2_ceil(pl.Rmax < 2 ? 2 : pl.Rmax);
        KSC_CUDA(cudaFuncSetAttribute(k_copy_cands, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
        k_copy_cands<<<(unsigned)nq, 256, csm, st>>>(topr, pl.Rmax, cand_out);
        ix->launches++;
        KSC_LAUNCH_CHECK();
    }
    if (!ids && !dists) {  // candidates only (a shard's first step): no re-rank
        mark(ix, KSC_NUM_STAGES, st);
        return KSC_OK;
    }
    // 6. exact rerank (precision variant: a BF16 / FP8 re-rank of the widened
    //    shortlist first, then FP32 of its best Rf), with the full queries and
    //    vectors (Alg. 2: q_init)
    mark(ix, 6, st);
    if (!Qr) Qr = Q;
    const float* Xr = rr_X(ix);
    const int dr = rr_d(ix);
    const uint64_t* rr_keys = topr;
    int rr_R = pl.Rmax;
    const int32_t* rr_q = pl.rerank_q;
    if (pl.prec > 0) {
        KSC_TRY(ensure_lowp(ix, pl.prec, st));
        KSC_TRY(ensure(ix->ws_topr2, sizeof(uint64_t) * nq * pl.Rf, st));
        uint64_t* topr2 = (uint64_t*)ix->ws_topr2.p;
        const size_t smem = sizeof(uint64_t) * pow2_ceil(pl.Rmax < 2 ? 2 : pl.Rmax);
        KSC_CUDA(cudaFuncSetAttribute(k_rerank_lowp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_rerank_lowp<<<(unsigned)nq, 256, smem, st>>>(Qr, dr, ix->metric == KSC_IP, pl.prec,
                                                       (const uint16_t*)ix->X_bf16, (const uint8_t*)ix->X_fp8,
                                                       ix->X_scale, topr, pl.Rmax, pl.rerank_q, pl.Rfix, pl.k, pl.Rf,
                                                       topr2);
        KSC_LAUNCH_CHECK();
        ix->launches++;
        rr_keys = topr2;
        rr_R = pl.Rf;
        rr_q = nullptr;
    }
    if (pl.k <= 32 && rr_R <= RW_MAXR && dr <= 128 && (dr & 3) == 0 && warp_per_query(nq)) {
        const bool band = pl.band && pl.prec == 0 && rr_R > pl.k;
        if (band) KSC_TRY(ensure_band(ix, st));
        const size_t smem = sizeof(uint64_t) * RW_WARPS * rr_R * (band ? 2 : 1) +
                            (band ? sizeof(uint32_t) * RW_WARPS * (rr_R + 64) : 0);
        auto kr = band && ix->x_u8_state == 1 ? k_rerank_w<true> : k_rerank_w<false>;
        KSC_CUDA(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kr<<<(unsigned)((nq + RW_WARPS - 1) / RW_WARPS), RW_WARPS * 32, smem, st>>>(
            Qr, Xr, dr, ix->metric == KSC_IP, rr_keys, rr_R, rr_q, rr_R, pl.k, nq, ids, dists,
            band && ix->x_u8_state != 1 ? (const uint16_t*)ix->X_bf16 : nullptr,
            band && ix->x_u8_state == 1 ? (const uint8_t*)ix->X_u8 : nullptr, band ? ix->X_band : nullptr);
        ix->launches++;
        KSC_LAUNCH_CHECK();
    } else {
        const size_t smem = sizeof(uint64_t) * pow2_ceil(rr_R < 2 ? 2 : rr_R);
        // a CTA per query; 1024 threads (more rows in flight) when the batch is
        // too small to fill the GPU with 256-thread CTAs
        if (nq < 2 * (int64_t)num_sms()) {
            KSC_CUDA(cudaFuncSetAttribute(k_rerank<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_rerank<1024><<<(unsigned)nq, 1024, smem, st>>>(Qr, Xr, dr, ix->metric == KSC_IP, rr_keys, rr_R, rr_q,
                                                             rr_R, pl.k, ids, dists);
        } else {
            KSC_CUDA(cudaFuncSetAttribute(k_rerank<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_rerank<256><<<(unsigned)nq, 256, smem, st>>>(Qr, Xr, dr, ix->metric == KSC_IP, rr_keys, rr_R, rr_q,
                                                           rr_R, pl.k, ids, dists);
        }
        ix->launches++;
        KSC_LAUNCH_CHECK();
    }
    mark(ix, KSC_NUM_STAGES, st);
    return KSC_OK;
}

// Tile lengths of the scan's warp items for an expected P probes per query.
// Short tiles balance the persistent warps, long ones amortise an item's
// set-up: about 220 items per SM for the filtered scan, and for the smaller
// unfiltered first part (its share from the split rule of k_count_parts:
// max(4 R, N / 16) keys, rounded up to whole lists) about 120, each within
// 4 to 32 blocks (on the 1M x 128 workload at nprobe 7: tiles of 14 and 6
// blocks; filtered tiles of 12 to 17 blocks ran within 1% of each other).
static void set_tiles(const ksc_index* ix, Plan& pl, int64_t nq, double P, const ksc_search_opts* opts) {
    const int QG = 32 / pl.G;
    const double nbar = (double)ix->n / ix->L;
    const double blocks = std::ceil((double)nq * P / ix->L / QG) * ix->nblocks;
    const double keys = std::max(P * nbar, 1.0);
    const double near =
        std::min(1.0, (std::max((double)NEAR_KEYS_PER_R * pl.Rmax, keys / NEAR_SHARE_DIV) + 0.5 * nbar) / keys);
    auto tile = [&](double b, double per_sm) {
        int t = (int)(b / (per_sm * num_sms()));
        t = t < 4 ? 4 : (t > 32 ? 32 : t);
        if (pl.G == 4) t = (t + S4_B - 1) / S4_B * S4_B;  // whole steps of 4 blocks
        return t;
    };
    pl.TB = tile(blocks * (1.0 - near), 220.0);
    pl.TBa = tile(blocks * near, 60.0);
    if (opts && opts->tile_blocks > 0) pl.TB = pl.TBa = std::min(opts->tile_blocks, 1 << 20);
    // tensor-core scan (the filtered part only): tiles of whole 128-vector
    // products, 32 blocks unless given
    if (pl.tc) pl.TB = (opts && opts->tile_blocks > 0) ? (std::min(opts->tile_blocks, 1 << 20) + 3) / 4 * 4 : 32;
}

static int make_plan(ksc_index* ix, int64_t nq, int k, int Pmax, int Rmax, const ksc_search_opts* opts, Plan& pl) {
    KSC_CHECK_ARG(nq >= 0, "nq < 0");
    KSC_CHECK_ARG(k >= 1 && k <= KSC_MAX_K, "k must be in [1, %d]", KSC_MAX_K);
    KSC_CHECK_ARG(Pmax >= 1 && Pmax <= ix->L && Pmax <= MAX_NPROBE, "nprobe must be in [1, min(nlist, %d)]",
                  MAX_NPROBE);
    if (Rmax < k) Rmax = k;
    KSC_CHECK_ARG(Rmax <= KSC_MAX_RERANK, "rerank must be <= %d", KSC_MAX_RERANK);
    pl.nq = nq;
    pl.k = k;
    pl.Pmax = Pmax;
    pl.Rmax = Rmax;
    pl.Pfix = Pmax;
    pl.Rfix = Rmax;
    pl.nprobe_q = nullptr;
    pl.rerank_q = nullptr;
    pl.G = choose_G(ix, nq, Pmax, opts ? opts->lanes_per_query : 0);
    pl.nt = tcs_nt(ix->M);
    pl.tc = opts && opts->scan_tc && !opts->hybrid && pl.nt > 0;
    set_tiles(ix, pl, nq, Pmax, opts);
    int cap = (opts && opts->cand_cap > 0) ? opts->cand_cap : std::max(32 * Rmax, 8192);
    pl.cap = std::max(cap, Rmax);
    pl.rank_mode = (opts && opts->rank_fp32) ? RANK_FP32 : ((opts && opts->rank_fp8) ? RANK_FP8 : RANK_TC16);
    pl.Pq_max = Pmax;
    pl.prec = opts ? opts->precision : 0;
    // the re-rank band: on by default for L2 (for inner products of
    // real-valued rows the BF16 band is wide against the gaps between the
    // best scores)
    pl.band = opts && opts->rerank_band != 0 ? opts->rerank_band > 0 : ix->metric != KSC_IP;
    KSC_CHECK_ARG(pl.prec >= 0 && pl.prec <= 2, "precision must be 0 (FP32), 1 (BF16) or 2 (FP8)");
    pl.Rf = pl.Rmax;
    if (pl.prec > 0) {
        const int rf = (opts->rerank_final > 0) ? opts->rerank_final : std::max(k, Rmax / 2);
        pl.Rf = std::min(std::max(rf, k), Rmax);
    }
    pl.hybrid = opts && opts->hybrid;
    pl.n_near = (opts && opts->n_near > 0) ? opts->n_near : 2;
    pl.efs = (opts && opts->efs > 0) ? opts->efs : 64;
    pl.tau = (opts && opts->tau >= 0 && opts->hybrid) ? opts->tau : 8;
    if (pl.hybrid) {
        KSC_CHECK_ARG(pl.efs <= 96, "efs must be <= 96");
        if (!ix->nbr_codes) {
            set_error("the hybrid search needs an index built or imported with graphs");
            return KSC_ESTATE;
        }
    }
    return KSC_OK;
}

}  // namespace ksc

using namespace ksc;

extern "C" {

int ksc_rank_lists(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t P, int32_t* probes_dev,
                   float* scores_dev, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    KSC_CHECK_ARG(P >= 1 && P <= ix->L && P <= MAX_NPROBE, "P must be in [1, min(nlist, %d)]", MAX_NPROBE);
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && probes_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    return rank_lists(ix, Qw, nq, nullptr, P, P, probes_dev, scores_dev, RANK_TC16, st);
}

int ksc_list_scores(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t tensor_cores, float* scores_dev,
                    float* err_dev, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && scores_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    KSC_CHECK_ARG(tensor_cores >= 0 && tensor_cores <= 2, "tensor_cores must be 0 (FP32), 1 (16-bit) or 2 (FP8)");
    const int mode = tensor_cores == 0 ? RANK_FP32 : (tensor_cores == 2 ? RANK_FP8 : RANK_TC16);
    float* err = nullptr;
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    KSC_TRY(list_scores(ix, Qw, nq, mode, scores_dev, &err, st));
    if (err_dev) KSC_CUDA(cudaMemcpyAsync(err_dev, err, sizeof(float) * nq, cudaMemcpyDeviceToDevice, st));
    return KSC_OK;
}

int ksc_compute_luts(ksc_index* ix, const float* Q_dev, int64_t nq, const int32_t* probes_dev, int32_t P,
                     uint8_t* lut_dev, int32_t* bias_dev, float* scale_dev, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    KSC_CHECK_ARG(P >= 1 && P <= ix->L, "P must be in [1, nlist]");
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && probes_dev && lut_dev && bias_dev && scale_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    return compute_luts(ix, Qw, nq, probes_dev, nullptr, P, P, lut_dev, bias_dev, scale_dev, st);
}

int ksc_search_with_probes(ksc_index* ix, const float* Q_dev, int64_t nq, const int32_t* probes_dev, int32_t P,
                           int32_t k, int32_t rerank, int64_t* ids_dev, float* dists_dev, uint64_t* cand_dev,
                           int32_t* ncand_dev, const ksc_search_opts* opts, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    Plan pl;
    KSC_TRY(make_plan(ix, nq, k, P, rerank, opts, pl));
    if (nq == 0) return KSC_OK;  // empty batch: pointers may be NULL
    KSC_CHECK_ARG(Q_dev && probes_dev && ids_dev && dists_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    KSC_CUDA(cudaMemsetAsync(ix->status, 0, sizeof(int32_t), st));
    KSC_CUDA(cudaMemsetAsync(ix->stats, 0, sizeof(unsigned long long) * 4, st));
    ix->launches = 0;
    mark(ix, 0, st);
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    return search_from_probes(ix, Qw, pl, probes_dev, ids_dev, dists_dev, cand_dev, ncand_dev, st, Q_dev);
}

}  // extern "C"

namespace ksc {
// A shard's first step (list sharding): steps a1 .. a5 with a fixed nprobe,
// the R = max(rerank, k) selected keys of every query, ascending, into
// keys [nq x R] (local ids; KEY_NONE pads a short list).
int search_keys(ksc_index* ix, const float* Q, int64_t nq, int nprobe, int rerank, const ksc_search_opts* opts,
                uint64_t* keys, cudaStream_t st) {
    Plan pl;
    KSC_TRY(make_plan(ix, nq, 1, nprobe, rerank, opts, pl));
    KSC_CHECK_ARG(!pl.hybrid && pl.prec == 0, "sharded search: plain scan and FP32 re-rank only");
    if (nq == 0) return KSC_OK;
    KSC_CUDA(cudaMemsetAsync(ix->status, 0, sizeof(int32_t), st));
    KSC_TRY(ensure(ix->ws_probes, sizeof(int32_t) * nq * pl.Pmax, st));
    int32_t* probes = (int32_t*)ix->ws_probes.p;
    KSC_CUDA(cudaMemsetAsync(ix->stats, 0, sizeof(unsigned long long) * 4, st));
    ix->launches = 0;
    mark(ix, 0, st);
    const float* Qw;
    KSC_TRY(work_queries(ix, Q, nq, st, &Qw));
    KSC_TRY(rank_lists(ix, Qw, nq, nullptr, pl.Pmax, pl.Pmax, probes, nullptr, pl.rank_mode, st));
    return search_from_probes(ix, Qw, pl, probes, nullptr, nullptr, keys, nullptr, st, Q);
}

// Exact re-rank (a6) of given candidate keys [nq x R] (local ids, KEY_NONE
// skipped): the k best by (distance, id) per query.
int rerank_keys(ksc_index* ix, const float* Q, int64_t nq, int k, const uint64_t* keys, int R, int64_t* ids,
                float* dists, cudaStream_t st) {
    const float* Xr = rr_X(ix);
    const int dr = rr_d(ix);
    const int ip = ix->metric == KSC_IP;
    if (k <= 32 && R <= RW_MAXR && dr <= 128 && (dr & 3) == 0 && warp_per_query(nq)) {
        const size_t smem = sizeof(uint64_t) * RW_WARPS * R;
        KSC_CUDA(cudaFuncSetAttribute(k_rerank_w<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_rerank_w<false><<<(unsigned)((nq + RW_WARPS - 1) / RW_WARPS), RW_WARPS * 32, smem, st>>>(
            Q, Xr, dr, ip, keys, R, nullptr, R, k, nq, ids, dists, nullptr, nullptr, nullptr);
    } else {
        const size_t smem = sizeof(uint64_t) * pow2_ceil(R < 2 ? 2 : R);
        if (nq < 2 * (int64_t)num_sms()) {
            KSC_CUDA(cudaFuncSetAttribute(k_rerank<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_rerank<1024><<<(unsigned)nq, 1024, smem, st>>>(Q, Xr, dr, ip, keys, R, nullptr, R, k, ids, dists);
        } else {
            KSC_CUDA(cudaFuncSetAttribute(k_rerank<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_rerank<256><<<(unsigned)nq, 256, smem, st>>>(Q, Xr, dr, ip, keys, R, nullptr, R, k, ids, dists);
        }
    }
    KSC_LAUNCH_CHECK();
    ix->launches++;
    return KSC_OK;
}
}  // namespace ksc

extern "C" {

int ksc_search(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, int32_t nprobe, int32_t rerank,
               int64_t* ids_dev, float* dists_dev, const ksc_search_opts* opts, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    Plan pl;
    KSC_TRY(make_plan(ix, nq, k, nprobe, rerank, opts, pl));
    if (nq == 0) return KSC_OK;  // empty batch: pointers may be NULL
    KSC_CHECK_ARG(Q_dev && ids_dev && dists_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    KSC_CUDA(cudaMemsetAsync(ix->status, 0, sizeof(int32_t), st));
    KSC_TRY(ensure(ix->ws_probes, sizeof(int32_t) * nq * pl.Pmax, st));
    int32_t* probes = (int32_t*)ix->ws_probes.p;
    KSC_CUDA(cudaMemsetAsync(ix->stats, 0, sizeof(unsigned long long) * 4, st));
    ix->launches = 0;
    mark(ix, 0, st);
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    KSC_TRY(rank_lists(ix, Qw, nq, nullptr, pl.Pmax, pl.Pmax, probes, nullptr, pl.rank_mode, st));
    return search_from_probes(ix, Qw, pl, probes, ids_dev, dists_dev, nullptr, nullptr, st, Q_dev);
}

int ksc_search_varprobe(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, const int32_t* nprobe_dev,
                        int32_t nprobe_max, const int32_t* rerank_dev, int32_t rerank_max, int64_t* ids_dev,
                        float* dists_dev, const ksc_search_opts* opts, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    Plan pl;
    KSC_TRY(make_plan(ix, nq, k, nprobe_max, rerank_max, opts, pl));
    if (nq == 0) return KSC_OK;  // empty batch: pointers may be NULL
    KSC_CHECK_ARG(Q_dev && ids_dev && dists_dev && nprobe_dev && rerank_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    pl.nprobe_q = nprobe_dev;
    pl.rerank_q = rerank_dev;
    set_tiles(ix, pl, nq, 0.5 * pl.Pmax, opts);  // per-query nprobe: about half the largest on average
    KSC_CUDA(cudaMemsetAsync(ix->status, 0, sizeof(int32_t), st));
    KSC_TRY(ensure(ix->ws_probes, sizeof(int32_t) * nq * pl.Pmax, st));
    int32_t* probes = (int32_t*)ix->ws_probes.p;
    KSC_CUDA(cudaMemsetAsync(ix->stats, 0, sizeof(unsigned long long) * 4, st));
    ix->launches = 0;
    mark(ix, 0, st);
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    KSC_TRY(rank_lists(ix, Qw, nq, nprobe_dev, pl.Pmax, pl.Pmax, probes, nullptr, pl.rank_mode, st));
    return search_from_probes(ix, Qw, pl, probes, ids_dev, dists_dev, nullptr, nullptr, st, Q_dev);
}

int ksc_profile_enable(ksc_index* ix, int32_t on) {
    KSC_CHECK_ARG(ix, "null argument");
    if (on) {
        for (int i = 0; i <= KSC_NUM_STAGES; ++i)
            if (!ix->ev[i]) KSC_CUDA(cudaEventCreate(&ix->ev[i]));
    }
    ix->prof = on != 0;
    for (int i = 0; i <= KSC_NUM_STAGES; ++i) ix->ev_used[i] = false;
    return KSC_OK;
}

int ksc_profile_read(ksc_index* ix, float* ms_host, int32_t n, int32_t* launches_host) {
    KSC_CHECK_ARG(ix && ms_host && n >= 0 && n <= 8, "bad argument");
    KSC_CHECK_ARG(ix->prof, "profiling is not enabled on this index");
    if (launches_host) *launches_host = ix->launches;
    for (int i = 0; i < n; ++i) ms_host[i] = 0.f;
    int prev = -1;
    for (int i = 0; i <= KSC_NUM_STAGES; ++i) {
        if (!ix->ev_used[i]) continue;
        KSC_CUDA(cudaEventSynchronize(ix->ev[i]));
        if (prev >= 0 && prev < n) {
            float ms = 0.f;
            KSC_CUDA(cudaEventElapsedTime(&ms, ix->ev[prev], ix->ev[i]));
            ms_host[prev] = ms;
        }
        prev = i;
    }
    return KSC_OK;
}

int ksc_lut16_peak(double* glookups_host, void* stream) {
    KSC_CHECK_ARG(glookups_host, "null argument");
    cudaStream_t st = as_stream(stream);
    uint32_t* sink = nullptr;
    KSC_CUDA(cudaMalloc(&sink, 16));
    const int iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // [0] the shared-selector sequence, 8 CTAs of 256 threads per SM;
    // [1] the per-slot sequence, 16 CTAs of 128 threads per SM
    double rate[2] = {0.0, 0.0};
    cudaError_t err = cudaSuccess;
    for (int v = 0; v < 2 && err == cudaSuccess; ++v) {
        const int threads = v == 0 ? 256 : 128, grid = num_sms() * (v == 0 ? 8 : 16);
        for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
            if (rep == 1) cudaEventRecord(e0, st);
            if (v == 0) k_lut16_peak_sel<<<grid, threads, 0, st>>>(iters, 12345u + rep, sink);
            else k_lut16_peak<<<grid, threads, 0, st>>>(iters, 12345u + rep, sink);
        }
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        rate[v] = (double)grid * threads * iters * 32 / (ms * 1e-3) / 1e9;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    KSC_CUDA(err);
    glookups_host[0] = rate[0];
    glookups_host[1] = rate[1];
    return KSC_OK;
}

int ksc_pair_distances(ksc_index* ix, const float* Q_dev, int64_t nq, const int64_t* ids_dev, int32_t c,
                       int32_t precision, float* out_dev, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    KSC_CHECK_ARG(precision >= 0 && precision <= 2, "precision must be 0, 1 or 2");
    if (nq == 0 || c == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && ids_dev && out_dev && c > 0, "bad argument");
    cudaStream_t st = as_stream(stream);
    KSC_TRY(ensure_lowp(ix, precision, st));
    k_pair_dist<<<(unsigned)nq, 256, 0, st>>>(Q_dev, nq, rr_d(ix), ix->metric == KSC_IP, precision, rr_X(ix),
                                              (const uint16_t*)ix->X_bf16, (const uint8_t*)ix->X_fp8, ix->X_scale,
                                              ids_dev, c, out_dev);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

int ksc_search_stats(ksc_index* ix, int64_t* stats_host) {
    KSC_CHECK_ARG(ix && stats_host, "null argument");
    unsigned long long v[4];
    KSC_CUDA(cudaMemcpy(v, ix->stats, sizeof(v), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; ++i) stats_host[i] = (int64_t)v[i];
    return KSC_OK;
}

int ksc_last_status(ksc_index* ix, int32_t* status_host) {
    KSC_CHECK_ARG(ix && status_host, "null argument");
    KSC_CUDA(cudaMemcpy(status_host, ix->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    return KSC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free LUT entry
// Some callers cannot let this library call cudaMalloc: a host program whose
// device memory is wholly reserved by its own allocator (a framework's caching
// pool, a serving runtime that pre-reserves the device) has no headroom for a
// foreign allocation, and a latency-critical caller cannot afford the device
// synchronisation that cudaMalloc / cudaFree may imply.  For them,
// ksc_compute_luts_noalloc keeps its only scratch -- the per-query table range
// that ksc_compute_luts otherwise keeps in a workspace buffer -- in the
// fixed-size array below.  Every GPU that loads the library holds the array
// (KSC_NOALLOC_MAX_NQ * 4 bytes = 256 KiB) until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_range[KSC_NOALLOC_MAX_NQ];

namespace ksc {
// Device address of g_noalloc_range per device ordinal, looked up on the first
// call made with that device current (host code cannot use the symbol itself:
// in host code it names a host-side stand-in, not device memory).  Atomic, so
// that host threads making their first call on one device at the same time
// do not race on the cache (they store the same address).
static std::atomic<void*> g_noalloc_addr[64] = {};
}  // namespace ksc

extern "C" int ksc_compute_luts_noalloc(ksc_index* ix, const float* Q_dev, int64_t nq, const int32_t* probes_dev,
                                        int32_t P, uint8_t* lut_dev, int32_t* bias_dev, float* scale_dev,
                                        void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    if (ix->dims) {
        set_error("ksc_compute_luts_noalloc needs an index without component filtration");
        return KSC_EUNSUPPORTED;
    }
    KSC_CHECK_ARG(P >= 1 && P <= ix->L, "P must be in [1, nlist]");
    KSC_CHECK_ARG(nq >= 0 && nq <= KSC_NOALLOC_MAX_NQ,
                  "nq = %lld exceeds the fixed scratch of ksc_compute_luts_noalloc (at most %d queries per call)",
                  (long long)nq, KSC_NOALLOC_MAX_NQ);
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && probes_dev && lut_dev && bias_dev && scale_dev, "null argument");
    int dev = 0;
    KSC_CUDA(cudaGetDevice(&dev));
    KSC_CHECK_ARG(dev >= 0 && dev < 64, "device ordinal %d out of range", dev);
    void* addr = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!addr) {
        KSC_CUDA(cudaGetSymbolAddress(&addr, g_noalloc_range));
        g_noalloc_addr[dev].store(addr, std::memory_order_release);
    }
    uint32_t* rb = static_cast<uint32_t*>(addr);
    cudaStream_t st = as_stream(stream);
    // the array keeps the previous call's ranges: clear this call's slots
    KSC_CUDA(cudaMemsetAsync(rb, 0, sizeof(uint32_t) * nq, st));
    LutArgs A{Q_dev, nq, ix->d, ix->M, ix->dsub, ix->metric == KSC_IP, P, probes_dev, nullptr, P, ix->c_mean,
              ix->codebook, ix->L};
    return launch_luts(A, rb, lut_dev, bias_dev, scale_dev, st);
}

// ------------------------------------------------------------------ learned nprobe / rerank
namespace ksc {
static const int32_t DEF_GRID[] = {4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128};
static const int32_t DEF_RGRID[] = {20, 50, 100, 200, 400};

// Rank with P probes (P >= 32) and derive the predictor features.
// The P best lists of every query (exact ranking) and the predictor's
// features, from the FEAT_K smallest given list scores (L >= FEAT_K).
static int rank_and_features(ksc_index* ix, const float* Q, int64_t nq, int P, int32_t* probes, float* feats,
                             cudaStream_t st) {
    KSC_TRY(ensure(ix->ws_rscore, sizeof(float) * nq * FEAT_K, st));
    float* rs = (float*)ix->ws_rscore.p;
    KSC_TRY(rank_lists(ix, Q, nq, nullptr, P, P, probes, nullptr, RANK_TC16, st, rs));
    KSC_TRY(mlp_features(rs, nq, FEAT_K, ix->spherical, feats, st));
    ix->launches++;
    return KSC_OK;
}

// The adaptive search's ranking (Sec. 4.2.1).  The predictor's distances
// are the FEAT_K smallest approximate list scores; the network sets each
// query's nprobe and R from them; only then are the nprobe best lists of each
// query ranked exactly, the threshold of the exact pass taken from the same
// sorted scores -- all in k_rank_head_w, with the CTA kernel for the queries
// it leaves on `redo`.  The probes equal the first nprobe of an exact ranking
// of Pr lists (an exact top-P is a prefix of the exact top-Pr); rows past
// nprobe hold -1.  Batches the warp kernels do not serve: the ranking of Pr
// lists with the features, then the head kernel.
static int rank_adaptive(ksc_index* ix, const float* Q, int64_t nq, int Pr, int32_t* probes,
                         const ksc_adaptive_params& prm, int32_t* np_q, int32_t* r_q, cudaStream_t st) {
    if (!rank_by_warp(ix, nq, Pr) || ix->L < FEAT_K) {
        KSC_TRY(ensure(ix->ws_rscore, sizeof(float) * nq * FEAT_K, st));
        float* rs = (float*)ix->ws_rscore.p;
        KSC_TRY(rank_lists(ix, Q, nq, nullptr, Pr, Pr, probes, nullptr, RANK_TC16, st, rs));
        KSC_TRY(mlp_infer_scores(ix->mlp_w, rs, FEAT_K, ix->spherical, nq, prm, np_q, r_q, st));
        ix->launches++;
        return KSC_OK;
    }
    KSC_TRY(ensure(ix->ws_scores, sizeof(float) * nq * ix->L, st));
    KSC_TRY(ensure(ix->ws_redo, sizeof(int32_t) * (nq + 1), st));
    float* scores = (float*)ix->ws_scores.p;
    int32_t* redo = (int32_t*)ix->ws_redo.p;
    float* err = nullptr;
    KSC_TRY(list_scores(ix, Q, nq, RANK_TC16, scores, &err, st));
    KSC_CUDA(cudaMemsetAsync(redo, 0, sizeof(int32_t), st));
    const size_t hsm = rh_head_bytes() + RH_WARPS * rh_warp_bytes(ix->L);
    KSC_CUDA(cudaFuncSetAttribute(k_rank_head_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
    int per_sm = 0;
    KSC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rank_head_w, RH_WARPS * 32, hsm));
    const int64_t grid = std::min<int64_t>((nq + RH_WARPS - 1) / RH_WARPS,
                                           (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1));
    k_rank_head_w<<<(unsigned)grid, RH_WARPS * 32, hsm, st>>>(scores, err, Q, ix->c_rank, nq, ix->d, ix->L,
                                                             ix->spherical, ix->mlp_w, prm, Pr, probes, redo, np_q,
                                                             r_q);
    KSC_LAUNCH_CHECK();
    // queries with too many lists inside the bound: the CTA kernel
    const int rs_cap = std::min(RS_CAP, std::max(1024, pow2_ceil(4 * Pr)));
    const size_t smem = rs_cap * sizeof(uint64_t) + (ix->L <= RS_SMEM_L ? sizeof(float) * ix->L : 0);
    KSC_CUDA(cudaFuncSetAttribute(k_rank_select<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_rank_select<256><<<num_sms() * 2, 256, smem, st>>>(scores, err, Q, ix->c_rank, nq, ix->d, ix->L, ix->spherical,
                                                        np_q, Pr, Pr, rs_cap, probes, nullptr, redo);
    KSC_LAUNCH_CHECK();
    ix->launches += 2;
    return KSC_OK;
}

static uint64_t mix64(uint64_t& s) {  // splitmix64 (Steele, Lea, Flood 2014)
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static float median_of(std::vector<int32_t> v) {
    if (v.empty()) return 0.f;
    std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
    return (float)v[v.size() / 2];
}

// Smallest grid value per query whose search finds >= target hits; queries
// that never reach it take the last grid value.
static int label_queries(ksc_index* ix, const float* Q, const float* Qr, int64_t nq, const float* kth,
                         const int32_t* probes, int Pr,
                         const std::vector<int32_t>& grid, bool over_rerank, const int32_t* nprobe_dev, int R_fixed,
                         int k, int target, std::vector<int32_t>& label, cudaStream_t st) {
    std::vector<int32_t> hits_h(nq);
    int32_t* hits = nullptr;
    int64_t* ids = nullptr;
    float* dists = nullptr;
    int32_t* cnst = nullptr;
    int rc = KSC_OK;
    label.assign(nq, -1);
    do {
        if (cudaMalloc(&hits, sizeof(int32_t) * nq) != cudaSuccess || cudaMalloc(&ids, sizeof(int64_t) * nq * k) != cudaSuccess ||
            cudaMalloc(&dists, sizeof(float) * nq * k) != cudaSuccess || cudaMalloc(&cnst, sizeof(int32_t) * nq) != cudaSuccess) {
            set_error("allocation failed while labelling");
            rc = KSC_ENOMEM;
            break;
        }
        for (int32_t gv : grid) {
            Plan pl;
            const int Rmax = over_rerank ? gv : R_fixed;
            if ((rc = make_plan(ix, nq, k, Pr, Rmax, nullptr, pl))) break;
            if (over_rerank) {
                pl.nprobe_q = nprobe_dev;
            } else {
                std::vector<int32_t> c(nq, gv);
                if (cudaMemcpy(cnst, c.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice) != cudaSuccess) {
                    rc = KSC_ECUDA;
                    break;
                }
                pl.nprobe_q = cnst;
            }
            if ((rc = search_from_probes(ix, Q, pl, probes, ids, dists, nullptr, nullptr, st, Qr))) break;
            if ((rc = mlp_hits(dists, nq, k, kth, ix->metric == KSC_IP, hits, st))) break;
            if (cudaMemcpyAsync(hits_h.data(), hits, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                set_error("label readback failed");
                rc = KSC_ECUDA;
                break;
            }
            for (int64_t q = 0; q < nq; ++q)
                if (label[q] < 0 && hits_h[q] >= target) label[q] = gv;
        }
    } while (0);
    for (auto& l : label)
        if (l < 0) l = grid.back();
    cudaFree(hits);
    cudaFree(ids);
    cudaFree(dists);
    cudaFree(cnst);
    return rc;
}
}  // namespace ksc

extern "C" {

int ksc_mlp_grad(const float* w_dev, const float* x_dev, const float* y_dev, int64_t B, float* grad_dev,
                 float* loss_dev, void* stream) {
    KSC_CHECK_ARG(w_dev && x_dev && y_dev && grad_dev && B > 0, "bad argument");
    return mlp_grad(w_dev, x_dev, y_dev, B, grad_dev, loss_dev, as_stream(stream));
}

int ksc_mlp_forward(const float* w_dev, const float* x_dev, int64_t B, float* prob_dev, void* stream) {
    KSC_CHECK_ARG(w_dev && x_dev && prob_dev && B > 0, "bad argument");
    ksc_adaptive_params prm = {1, 1, 1, 1, 0.f, 0.f, 0.f, 0.f};
    return mlp_infer(w_dev, x_dev, B, prm, prob_dev, nullptr, nullptr, as_stream(stream));
}

int ksc_query_features(ksc_index* ix, const float* Q_dev, int64_t nq, float* feats_dev, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    KSC_CHECK_ARG(ix->L >= 32, "the predictor needs at least 32 lists");
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && feats_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    KSC_TRY(ensure(ix->ws_probes, sizeof(int32_t) * nq, st));
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    return rank_and_features(ix, Qw, nq, 1, (int32_t*)ix->ws_probes.p, feats_dev, st);
}

int ksc_predictor_params(ksc_index* ix, const ksc_adaptive_params* prm) {
    KSC_CHECK_ARG(ix && prm, "null argument");
    KSC_CHECK_ARG(prm->pmin >= 1 && prm->pmin <= prm->pmax && prm->pmax <= ix->L && prm->pmax <= MAX_NPROBE,
                  "nprobe range must satisfy 1 <= pmin <= pmax <= min(nlist, %d)", MAX_NPROBE);
    KSC_CHECK_ARG(prm->rmin >= 1 && prm->rmin <= prm->rmax && prm->rmax <= KSC_MAX_RERANK, "bad rerank range");
    ix->mlp_prm = *prm;
    return KSC_OK;
}

int ksc_predictor_weights(ksc_index* ix, float* w_host, const float* w_in_host) {
    KSC_CHECK_STATE(!ix || !w_in_host || !ix->parent, "models are set on the index, not on a view of it");
    KSC_CHECK_ARG(ix && (w_host || w_in_host), "null argument");
    if (w_in_host) {
        if (!ix->mlp_w) KSC_CUDA(cudaMalloc(&ix->mlp_w, sizeof(float) * KSC_MLP_NPARAMS));
        KSC_CUDA(cudaMemcpy(ix->mlp_w, w_in_host, sizeof(float) * KSC_MLP_NPARAMS, cudaMemcpyHostToDevice));
        if (ix->mlp_prm.pmax == 0) {
            ix->mlp_prm = {DEF_GRID[0], std::min(DEF_GRID[10], ix->L), DEF_RGRID[0], DEF_RGRID[4], 0.3f, 0.5f,
                           0.3f, 0.5f};
            if (ix->mlp_prm.pmin > ix->mlp_prm.pmax) ix->mlp_prm.pmin = ix->mlp_prm.pmax;
        }
    }
    if (w_host) {
        if (!ix->mlp_w) {
            set_error("no predictor has been trained or loaded");
            return KSC_ESTATE;
        }
        KSC_CUDA(cudaMemcpy(w_host, ix->mlp_w, sizeof(float) * KSC_MLP_NPARAMS, cudaMemcpyDeviceToHost));
    }
    return KSC_OK;
}

int ksc_train_predictor(ksc_index* ix, const float* Qtrain_dev, int64_t nt, const float* kth_dev,
                        const ksc_train_opts* opts, void* stream, float* loss_host) {
    KSC_CHECK_STATE(!ix || !ix->parent, "the predictor is trained on an index, not on a view of it");
    KSC_CHECK_ARG(ix && Qtrain_dev && kth_dev && nt > 0, "bad argument");
    KSC_CHECK_ARG(ix->L >= 32, "the predictor needs at least 32 lists");
    cudaStream_t st = as_stream(stream);
    const int k = (opts && opts->k > 0) ? opts->k : 10;
    const int target = (opts && opts->target_hits > 0) ? opts->target_hits : 9;
    const int R_lab = (opts && opts->rerank_label > 0) ? opts->rerank_label : 200;
    const int epochs = (opts && opts->epochs > 0) ? opts->epochs : 8;
    const int batch = (opts && opts->batch > 0) ? opts->batch : 256;
    const float lr = (opts && opts->lr > 0.f) ? opts->lr : 1e-3f;
    uint64_t seed = (opts && opts->seed) ? opts->seed : 0x6d6c70ull;
    const bool regression = opts && opts->regression;
    std::vector<int32_t> grid, rgrid;
    if (opts && opts->grid_host && opts->ngrid > 0) grid.assign(opts->grid_host, opts->grid_host + opts->ngrid);
    else grid.assign(DEF_GRID, DEF_GRID + 11);
    if (opts && opts->rgrid_host && opts->nrgrid > 0) rgrid.assign(opts->rgrid_host, opts->rgrid_host + opts->nrgrid);
    else rgrid.assign(DEF_RGRID, DEF_RGRID + 5);
    while (!grid.empty() && grid.back() > ix->L) grid.pop_back();
    KSC_CHECK_ARG(!grid.empty() && !rgrid.empty(), "empty grid");
    KSC_CHECK_ARG(rgrid.back() <= KSC_MAX_RERANK && R_lab >= k, "bad rerank grid");
    const int Pr = std::min(std::max(grid.back(), 32), ix->L);
    const int64_t chunk = 8192;
    float* feats = nullptr;
    float* Y = nullptr;
    int32_t* probes = nullptr;
    int32_t* lab_dev = nullptr;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *xb = nullptr, *yb = nullptr, *lossd = nullptr;
    int64_t* idx = nullptr;
    std::vector<int32_t> lab_n(nt), lab_r(nt);
    int rc = KSC_OK;
    const int steps = (int)((nt + batch - 1) / batch);
#define T_CUDA(call) { cudaError_t e_ = (call); if (e_ != cudaSuccess) { set_error("%s: %s", #call, cudaGetErrorString(e_)); rc = KSC_ECUDA; break; } }
    do {
        T_CUDA(cudaMalloc(&feats, sizeof(float) * nt * KSC_MLP_FEATURES));
        T_CUDA(cudaMalloc(&Y, sizeof(float) * nt * 2));
        T_CUDA(cudaMalloc(&probes, sizeof(int32_t) * chunk * Pr));
        T_CUDA(cudaMalloc(&lab_dev, sizeof(int32_t) * chunk));
        // 1. labels from the plain search, chunk by chunk
        for (int64_t c0 = 0; c0 < nt && rc == KSC_OK; c0 += chunk) {
            const int64_t nc = std::min(chunk, nt - c0);
            const float* Qc = Qtrain_dev + c0 * rr_d(ix);
            const float* Qcw;
            if ((rc = work_queries(ix, Qc, nc, st, &Qcw))) break;
            if ((rc = rank_and_features(ix, Qcw, nc, Pr, probes, feats + c0 * KSC_MLP_FEATURES, st))) break;
            std::vector<int32_t> ln, lr_;
            if ((rc = label_queries(ix, Qcw, Qc, nc, kth_dev + c0, probes, Pr, grid, false, nullptr, R_lab, k, target,
                                    ln, st)))
                break;
            T_CUDA(cudaMemcpy(lab_dev, ln.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice));
            if ((rc = label_queries(ix, Qcw, Qc, nc, kth_dev + c0, probes, Pr, rgrid, true, lab_dev, 0, k, target,
                                    lr_, st)))
                break;
            std::copy(ln.begin(), ln.end(), lab_n.begin() + c0);
            std::copy(lr_.begin(), lr_.end(), lab_r.begin() + c0);
        }
        if (rc) break;
        const float med_n = median_of(lab_n), med_r = median_of(lab_r);
        std::vector<float> yh(nt * 2);
        // regression heads: soft targets, the normalised log of the label
        auto soft = [](int32_t v, int32_t lo, int32_t hi) {
            return hi > lo ? (float)((std::log((double)v) - std::log((double)lo)) / (std::log((double)hi) - std::log((double)lo)))
                           : 0.f;
        };
        for (int64_t q = 0; q < nt; ++q) {
            if (regression) {
                yh[2 * q] = soft(lab_n[q], grid.front(), grid.back());
                yh[2 * q + 1] = soft(lab_r[q], rgrid.front(), rgrid.back());
            } else {
                yh[2 * q] = lab_n[q] > med_n ? 1.f : 0.f;
                yh[2 * q + 1] = lab_r[q] > med_r ? 1.f : 0.f;
            }
        }
        T_CUDA(cudaMemcpy(Y, yh.data(), sizeof(float) * nt * 2, cudaMemcpyHostToDevice));
        // 2. weights: He-uniform from the seed, zero biases
        std::vector<float> wh(KSC_MLP_NPARAMS, 0.f);
        const int fan[3] = {KSC_MLP_FEATURES, 64, 64}, rows[3] = {64, 64, 2};
        int off = 0;
        for (int l = 0; l < 3; ++l) {
            const float a = sqrtf(6.f / fan[l]);
            for (int e = 0; e < rows[l] * fan[l]; ++e)
                wh[off + e] = a * (2.f * (float)((mix64(seed) >> 11) * (1.0 / 9007199254740992.0)) - 1.f);
            off += rows[l] * fan[l] + rows[l];
        }
        T_CUDA(cudaMalloc(&w, sizeof(float) * KSC_MLP_NPARAMS));
        T_CUDA(cudaMalloc(&g, sizeof(float) * KSC_MLP_NPARAMS));
        T_CUDA(cudaMalloc(&m, sizeof(float) * KSC_MLP_NPARAMS));
        T_CUDA(cudaMalloc(&v, sizeof(float) * KSC_MLP_NPARAMS));
        T_CUDA(cudaMalloc(&xb, sizeof(float) * batch * KSC_MLP_FEATURES));
        T_CUDA(cudaMalloc(&yb, sizeof(float) * batch * 2));
        T_CUDA(cudaMalloc(&idx, sizeof(int64_t) * nt));
        T_CUDA(cudaMalloc(&lossd, sizeof(float) * steps));
        T_CUDA(cudaMemcpy(w, wh.data(), sizeof(float) * KSC_MLP_NPARAMS, cudaMemcpyHostToDevice));
        T_CUDA(cudaMemset(m, 0, sizeof(float) * KSC_MLP_NPARAMS));
        T_CUDA(cudaMemset(v, 0, sizeof(float) * KSC_MLP_NPARAMS));
        // 3. Adam over shuffled minibatches
        std::vector<int64_t> perm(nt);
        int t = 0;
        for (int ep = 0; ep < epochs && rc == KSC_OK; ++ep) {
            for (int64_t i = 0; i < nt; ++i) perm[i] = i;
            for (int64_t i = nt - 1; i > 0; --i) std::swap(perm[i], perm[(int64_t)(mix64(seed) % (uint64_t)(i + 1))]);
            T_CUDA(cudaMemcpyAsync(idx, perm.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, st));
            for (int s_ = 0; s_ < steps; ++s_) {
                const int64_t b0 = (int64_t)s_ * batch, nb = std::min<int64_t>(batch, nt - b0);
                k_gather_rows<<<(unsigned)((nb * KSC_MLP_FEATURES + 255) / 256), 256, 0, st>>>(feats, idx + b0, nb,
                                                                                             KSC_MLP_FEATURES, xb);
                k_gather_rows<<<(unsigned)((nb * 2 + 255) / 256), 256, 0, st>>>(Y, idx + b0, nb, 2, yb);
                if ((rc = mlp_grad(w, xb, yb, nb, g, lossd + s_, st))) break;
                if ((rc = mlp_adam(w, g, m, v, ++t, lr, st))) break;
            }
            T_CUDA(cudaStreamSynchronize(st));  // perm is reused by the next epoch
        }
        if (rc) break;
        if (loss_host) {
            std::vector<float> lh(steps);
            T_CUDA(cudaMemcpy(lh.data(), lossd, sizeof(float) * steps, cudaMemcpyDeviceToHost));
            double sum = 0.0;
            for (float x : lh) sum += x;
            *loss_host = (float)(sum / steps);
        }
        if (ix->mlp_w) cudaFree(ix->mlp_w);
        ix->mlp_w = w;
        w = nullptr;
        ix->mlp_prm = regression
                          ? ksc_adaptive_params{grid.front(), grid.back(), rgrid.front(), rgrid.back(), 0.f, 0.f, 0.f,
                                                0.f, 1}
                          : ksc_adaptive_params{grid.front(), grid.back(), rgrid.front(), rgrid.back(), 0.3f, 0.5f,
                                                0.3f, 0.5f, 0};
    } while (0);
#undef T_CUDA
    cudaFree(feats); cudaFree(Y); cudaFree(probes); cudaFree(lab_dev); cudaFree(w); cudaFree(g); cudaFree(m);
    cudaFree(v); cudaFree(xb); cudaFree(yb); cudaFree(idx); cudaFree(lossd);
    return rc;
}

int ksc_search_adaptive(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, int64_t* ids_dev,
                        float* dists_dev, int32_t* nprobe_dev, int32_t* rerank_dev, const ksc_search_opts* opts,
                        void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    if (!ix->mlp_w) {
        set_error("no predictor has been trained or loaded");
        return KSC_ESTATE;
    }
    const ksc_adaptive_params& prm = ix->mlp_prm;
    const int Pr = std::min(std::max(prm.pmax, 1), ix->L);  // the lists a query may probe
    Plan pl;
    KSC_TRY(make_plan(ix, nq, k, Pr, prm.rmax, opts, pl));
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && ids_dev && dists_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    KSC_CUDA(cudaMemsetAsync(ix->status, 0, sizeof(int32_t), st));
    KSC_CUDA(cudaMemsetAsync(ix->stats, 0, sizeof(unsigned long long) * 4, st));
    KSC_TRY(ensure(ix->ws_probes, sizeof(int32_t) * nq * Pr, st));
    KSC_TRY(ensure(ix->ws_nprobe, sizeof(int32_t) * nq, st));
    KSC_TRY(ensure(ix->ws_rerank, sizeof(int32_t) * nq, st));
    int32_t* probes = (int32_t*)ix->ws_probes.p;
    int32_t* np_q = (int32_t*)ix->ws_nprobe.p;
    int32_t* r_q = (int32_t*)ix->ws_rerank.p;
    ix->launches = 0;
    mark(ix, 0, st);
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    KSC_TRY(rank_adaptive(ix, Qw, nq, Pr, probes, prm, np_q, r_q, st));
    pl.nprobe_q = np_q;
    pl.rerank_q = r_q;
    pl.Pq_max = std::min(prm.pmax, Pr);
    const int32_t* sprobes = probes;
    if (ix->pr_theta >= 0.f && ix->pr_model && ix->pr_have_stats) {
        // Alg. 2: predictive pruning of the predicted nprobe lists
        KSC_TRY(ensure(ix->ws_pprobes, sizeof(int32_t) * nq * Pr, st));
        KSC_TRY(ensure(ix->ws_pn, sizeof(int32_t) * nq, st));
        int32_t* kept = (int32_t*)ix->ws_pprobes.p;
        int32_t* pn = (int32_t*)ix->ws_pn.p;
        KSC_TRY(prune_rows(ix, Qw, nq, probes, Pr, np_q, Pr, ix->pr_theta, nullptr, nullptr, kept, pn, st));
        ix->launches += 2;
        sprobes = kept;
        np_q = pn;
        pl.nprobe_q = pn;
    }
    set_tiles(ix, pl, nq, 0.5 * (prm.pmin + prm.pmax), opts);
    KSC_TRY(search_from_probes(ix, Qw, pl, sprobes, ids_dev, dists_dev, nullptr, nullptr, st, Q_dev));
    if (nprobe_dev) KSC_CUDA(cudaMemcpyAsync(nprobe_dev, np_q, sizeof(int32_t) * nq, cudaMemcpyDeviceToDevice, st));
    if (rerank_dev) KSC_CUDA(cudaMemcpyAsync(rerank_dev, r_q, sizeof(int32_t) * nq, cudaMemcpyDeviceToDevice, st));
    return KSC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ captured plans, autotuner
struct ksc_plan {
    ksc_index* ix = nullptr;
    int64_t nq = 0;
    int32_t k = 0, nprobe = 0, rerank = 0, adaptive = 0;
    ksc_search_opts opts = {};
    bool has_opts = false;
    float* Q = nullptr;
    int64_t* ids = nullptr;
    float* dists = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long gen = 0;
};

namespace ksc {
static int plan_search(ksc_plan* pl, cudaStream_t st) {
    const ksc_search_opts* o = pl->has_opts ? &pl->opts : nullptr;
    if (pl->adaptive)
        return ksc_search_adaptive(pl->ix, pl->Q, pl->nq, pl->k, pl->ids, pl->dists, nullptr, nullptr, o, st);
    return ksc_search(pl->ix, pl->Q, pl->nq, pl->k, pl->nprobe, pl->rerank, pl->ids, pl->dists, o, st);
}

// Warm the workspace with one search, then capture the next into a graph.
static int plan_capture(ksc_plan* pl, cudaStream_t st) {
    if (pl->exec) { cudaGraphExecDestroy(pl->exec); pl->exec = nullptr; }
    if (pl->graph) { cudaGraphDestroy(pl->graph); pl->graph = nullptr; }
    const bool prof = pl->ix->prof;
    pl->ix->prof = false;
    int rc = plan_search(pl, st);
    if (rc == KSC_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { set_error("warm-up failed: %s", cudaGetErrorString(e)); rc = KSC_ECUDA; }
    }
    if (rc == KSC_OK) {
        pl->gen = workspace_generation();
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            set_error("stream capture failed to start: %s", cudaGetErrorString(e));
            rc = KSC_ECUDA;
        } else {
            rc = plan_search(pl, st);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(st, &g);
            if (rc == KSC_OK && e != cudaSuccess) {
                set_error("stream capture failed: %s", cudaGetErrorString(e));
                rc = KSC_ECUDA;
            }
            pl->graph = g;
            if (rc == KSC_OK && workspace_generation() != pl->gen) {
                set_error("workspace changed during capture");
                rc = KSC_ESTATE;
            }
            if (rc == KSC_OK) {
                e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
                if (e != cudaSuccess) {
                    set_error("graph instantiation failed: %s", cudaGetErrorString(e));
                    rc = KSC_ECUDA;
                }
            }
        }
    }
    pl->ix->prof = prof;
    return rc;
}
}  // namespace ksc

extern "C" {

void ksc_plan_free(ksc_plan* pl) {
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    cudaFree(pl->Q);
    cudaFree(pl->ids);
    cudaFree(pl->dists);
    delete pl;
}

int ksc_plan_create(ksc_index* ix, int64_t nq, int32_t k, int32_t nprobe, int32_t rerank, int32_t adaptive,
                    const ksc_search_opts* opts, void* stream, ksc_plan** out) {
    KSC_CHECK_ARG(ix && out && nq > 0 && k >= 1, "bad argument");
    KSC_CHECK_ARG(stream != nullptr, "plans need a non-default stream (graph capture)");
    cudaStream_t st = as_stream(stream);
    ksc_plan* pl = new ksc_plan();
    pl->ix = ix;
    pl->nq = nq;
    pl->k = k;
    pl->nprobe = nprobe;
    pl->rerank = rerank;
    pl->adaptive = adaptive;
    if (opts) { pl->opts = *opts; pl->has_opts = true; }
    int rc = KSC_OK;
    if (cudaMalloc(&pl->Q, sizeof(float) * nq * rr_d(ix)) != cudaSuccess ||
        cudaMalloc(&pl->ids, sizeof(int64_t) * nq * k) != cudaSuccess ||
        cudaMalloc(&pl->dists, sizeof(float) * nq * k) != cudaSuccess) {
        set_error("plan buffer allocation failed");
        rc = KSC_ENOMEM;
    }
    if (rc == KSC_OK && cudaMemsetAsync(pl->Q, 0, sizeof(float) * nq * rr_d(ix), st) != cudaSuccess) rc = KSC_ECUDA;
    if (rc == KSC_OK) rc = plan_capture(pl, st);
    if (rc != KSC_OK) {
        ksc_plan_free(pl);
        return rc;
    }
    *out = pl;
    return KSC_OK;
}

int ksc_plan_buffers(ksc_plan* pl, float** Q_dev, int64_t** ids_dev, float** dists_dev) {
    KSC_CHECK_ARG(pl, "null plan");
    if (Q_dev) *Q_dev = pl->Q;
    if (ids_dev) *ids_dev = pl->ids;
    if (dists_dev) *dists_dev = pl->dists;
    return KSC_OK;
}

int ksc_plan_execute(ksc_plan* pl, const float* Q_dev, int64_t* ids_dev, float* dists_dev, void* stream) {
    KSC_CHECK_ARG(pl && pl->exec, "null plan");
    cudaStream_t st = as_stream(stream);
    KSC_CHECK_ARG(stream != nullptr, "plans need a non-default stream (graph capture)");
    if (Q_dev && Q_dev != pl->Q)
        KSC_CUDA(cudaMemcpyAsync(pl->Q, Q_dev, sizeof(float) * pl->nq * rr_d(pl->ix), cudaMemcpyDeviceToDevice, st));
    if (workspace_generation() != pl->gen) KSC_TRY(plan_capture(pl, st));
    KSC_CUDA(cudaGraphLaunch(pl->exec, st));
    if (ids_dev && ids_dev != pl->ids)
        KSC_CUDA(cudaMemcpyAsync(ids_dev, pl->ids, sizeof(int64_t) * pl->nq * pl->k, cudaMemcpyDeviceToDevice, st));
    if (dists_dev && dists_dev != pl->dists)
        KSC_CUDA(cudaMemcpyAsync(dists_dev, pl->dists, sizeof(float) * pl->nq * pl->k, cudaMemcpyDeviceToDevice, st));
    return KSC_OK;
}

int ksc_autotune(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, int32_t nprobe, int32_t rerank,
                 ksc_search_opts* opts, void* stream, float* best_ms_host) {
    KSC_CHECK_ARG(ix && Q_dev && opts && nq > 0, "bad argument");
    cudaStream_t st = as_stream(stream);
    int64_t* ids = nullptr;
    float* dists = nullptr;
    KSC_CUDA(cudaMalloc(&ids, sizeof(int64_t) * nq * k));
    cudaError_t ea = cudaMalloc(&dists, sizeof(float) * nq * k);
    if (ea != cudaSuccess) { cudaFree(ids); KSC_CUDA(ea); }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int Gs[4] = {4, 8, 16, 32};
    const int TBs[5] = {0, 8, 16, 32, 64};
    ksc_search_opts best = *opts;
    float best_ms = INFINITY;
    int rc = KSC_OK;
    for (int gi = 0; gi < 4 && rc == KSC_OK; ++gi) {
        if (Gs[gi] == 4 ? ix->M > 128 : (ix->M + Gs[gi] - 1) / Gs[gi] > 16) continue;
        for (int ti = 0; ti < 5 && rc == KSC_OK; ++ti) {
            ksc_search_opts o = *opts;
            o.lanes_per_query = Gs[gi];
            o.tile_blocks = TBs[ti];
            float ms = 0.f, tot = 0.f;
            for (int rep = 0; rep < 4 && rc == KSC_OK; ++rep) {
                cudaEventRecord(e0, st);
                rc = ksc_search(ix, Q_dev, nq, k, nprobe, rerank, ids, dists, &o, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) { set_error("autotune run failed"); rc = KSC_ECUDA; }
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep >= 1) tot += ms;  // the first run warms the workspace
            }
            if (rc == KSC_OK && tot / 3 < best_ms) {
                best_ms = tot / 3;
                best = o;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ids);
    cudaFree(dists);
    if (rc != KSC_OK) return rc;
    opts->lanes_per_query = best.lanes_per_query;
    opts->tile_blocks = best.tile_blocks;
    if (best_ms_host) *best_ms_host = best_ms;
    return KSC_OK;
}

}  // extern "C"


// ------------------------------------------------------------------ predictive cluster pruning
// Sec. 4.2.3, Table 4, Alg. 2 f_prune: statistics, features and the
// classifier live in prune.cu; here are the entry points that tie them to the
// ranking, the plain search (labels) and the search of the kept lists.
extern "C" {

int ksc_pruner_stats(ksc_index* ix, int32_t iters, void* stream) {
    KSC_CHECK_STATE(!ix || !ix->parent, "the pruning statistics belong to the index, not to a view of it");
    KSC_CHECK_ARG(ix, "null index");
    return prune_stats(ix, iters, as_stream(stream));
}

int ksc_pruner_export(ksc_index* ix, float* stats_host, float* vecs_host, float* model_host) {
    KSC_CHECK_ARG(ix, "null index");
    if (stats_host || vecs_host) KSC_CHECK_STATE(ix->pr_have_stats, "the pruning statistics have not been computed");
    if (model_host) KSC_CHECK_STATE(ix->pr_model, "no pruning model");
    KSC_CUDA(cudaDeviceSynchronize());
    if (stats_host)
        KSC_CUDA(cudaMemcpy(stats_host, ix->pr_stats, sizeof(float) * ix->L * KSC_PRUNE_STATS, cudaMemcpyDeviceToHost));
    if (vecs_host)
        KSC_CUDA(cudaMemcpy(vecs_host, ix->pr_vecs, sizeof(float) * ix->L * 3 * ix->d, cudaMemcpyDeviceToHost));
    if (model_host)
        KSC_CUDA(cudaMemcpy(model_host, ix->pr_model, sizeof(float) * KSC_PRUNE_MODEL, cudaMemcpyDeviceToHost));
    return KSC_OK;
}

int ksc_pruner_import_model(ksc_index* ix, const float* model_host) {
    KSC_CHECK_STATE(!ix || !ix->parent, "models are set on the index, not on a view of it");
    KSC_CHECK_ARG(ix && model_host, "null argument");
    if (!ix->pr_model) KSC_CUDA(cudaMalloc(&ix->pr_model, sizeof(float) * KSC_PRUNE_MODEL));
    KSC_CUDA(cudaMemcpy(ix->pr_model, model_host, sizeof(float) * KSC_PRUNE_MODEL, cudaMemcpyHostToDevice));
    bump_workspace_generation();
    return KSC_OK;
}

int ksc_pruner_theta(ksc_index* ix, float theta) {
    KSC_CHECK_ARG(ix, "null index");
    KSC_CHECK_STATE(theta < 0.f || (ix->pr_have_stats && ix->pr_model), "no pruning model");
    ix->pr_theta = theta;
    bump_workspace_generation();
    return KSC_OK;
}

int ksc_prune_probes(ksc_index* ix, const float* Q_dev, int64_t nq, const int32_t* probes_dev, int32_t Pmax,
                     const int32_t* nprobe_dev, int32_t P, float theta, float* feats_dev, float* prob_dev,
                     int32_t* probes_out_dev, int32_t* nprobe_out_dev, void* stream) {
    KSC_CHECK_ARG(ix && nq >= 0 && Pmax >= 1 && (nprobe_dev || (P >= 1 && P <= Pmax)), "bad argument");
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && probes_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    return prune_rows(ix, Qw, nq, probes_dev, Pmax, nprobe_dev, P, theta, feats_dev, prob_dev, probes_out_dev,
                      nprobe_out_dev, st);
}

int ksc_prune_labels(ksc_index* ix, const int64_t* ids_dev, const float* dists_dev, int64_t nq, int32_t k,
                     const float* kth_dev, const int32_t* probes_dev, int32_t Pmax, int32_t P, float* label_dev,
                     void* stream) {
    KSC_CHECK_ARG(ix && nq >= 0 && k >= 1 && Pmax >= 1 && P >= 0, "bad argument");
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(ids_dev && dists_dev && kth_dev && probes_dev && label_dev, "null argument");
    return prune_labels(ix, ids_dev, dists_dev, nq, k, kth_dev, probes_dev, Pmax, P, label_dev, as_stream(stream));
}

int ksc_prune_mlp_grad(const float* w_dev, const float* x_dev, const float* y_dev, int64_t B, float* grad_dev,
                       float* loss_dev, void* stream) {
    KSC_CHECK_ARG(w_dev && x_dev && y_dev && grad_dev && B > 0, "bad argument");
    return prune_mlp_grad(w_dev, x_dev, y_dev, B, grad_dev, loss_dev, as_stream(stream));
}

int ksc_search_pruned(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, int32_t nprobe, int32_t rerank,
                      float theta, int64_t* ids_dev, float* dists_dev, int32_t* nprobe_out_dev,
                      const ksc_search_opts* opts, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    KSC_CHECK_STATE(ix->pr_have_stats && ix->pr_model, "no pruning model: train one with ksc_train_pruner");
    Plan pl;
    KSC_TRY(make_plan(ix, nq, k, nprobe, rerank, opts, pl));
    if (nq == 0) return KSC_OK;  // empty batch: pointers may be NULL
    KSC_CHECK_ARG(Q_dev && ids_dev && dists_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    KSC_CUDA(cudaMemsetAsync(ix->status, 0, sizeof(int32_t), st));
    KSC_TRY(ensure(ix->ws_probes, sizeof(int32_t) * nq * pl.Pmax, st));
    KSC_TRY(ensure(ix->ws_pprobes, sizeof(int32_t) * nq * pl.Pmax, st));
    KSC_TRY(ensure(ix->ws_pn, sizeof(int32_t) * nq, st));
    int32_t* probes = (int32_t*)ix->ws_probes.p;
    int32_t* kept = (int32_t*)ix->ws_pprobes.p;
    int32_t* pn = (int32_t*)ix->ws_pn.p;
    KSC_CUDA(cudaMemsetAsync(ix->stats, 0, sizeof(unsigned long long) * 4, st));
    ix->launches = 0;
    mark(ix, 0, st);
    const float* Qw;
    KSC_TRY(work_queries(ix, Q_dev, nq, st, &Qw));
    KSC_TRY(rank_lists(ix, Qw, nq, nullptr, pl.Pmax, pl.Pmax, probes, nullptr, pl.rank_mode, st));
    // Alg. 2: keep rank 0 and the ranks with f_prune > theta, in rank order
    KSC_TRY(prune_rows(ix, Qw, nq, probes, pl.Pmax, nullptr, pl.Pmax, theta, nullptr, nullptr, kept, pn, st));
    ix->launches++;
    pl.nprobe_q = pn;
    set_tiles(ix, pl, nq, 0.75 * pl.Pmax, opts);
    if (nprobe_out_dev)
        KSC_CUDA(cudaMemcpyAsync(nprobe_out_dev, pn, sizeof(int32_t) * nq, cudaMemcpyDeviceToDevice, st));
    return search_from_probes(ix, Qw, pl, kept, ids_dev, dists_dev, nullptr, nullptr, st, Q_dev);
}

#define T_CUDA(call) { cudaError_t e_ = (call); if (e_ != cudaSuccess) { set_error("%s: %s", #call, cudaGetErrorString(e_)); rc = KSC_ECUDA; break; } }
int ksc_train_pruner(ksc_index* ix, const float* Qtrain_dev, int64_t nt, const float* kth_dev, int32_t k,
                     int32_t P, int32_t R, const ksc_train_opts* opts, void* stream, float* loss_host) {
    KSC_CHECK_STATE(!ix || !ix->parent, "the pruner is trained on an index, not on a view of it");
    KSC_CHECK_ARG(ix && Qtrain_dev && kth_dev && nt > 0, "bad argument");
    KSC_CHECK_ARG(k >= 1 && k <= KSC_MAX_K && R >= k && R <= KSC_MAX_RERANK, "bad k or rerank");
    KSC_CHECK_ARG(P >= 1 && P <= ix->L && P <= MAX_NPROBE, "bad nprobe");
    cudaStream_t st = as_stream(stream);
    if (!ix->pr_have_stats) KSC_TRY(prune_stats(ix, 30, st));
    const int epochs = (opts && opts->epochs > 0) ? opts->epochs : 4;
    const int batch = (opts && opts->batch > 0) ? opts->batch : 1024;
    const float lr = (opts && opts->lr > 0.f) ? opts->lr : 1e-3f;
    uint64_t seed = (opts && opts->seed) ? opts->seed : 0x707275ull;
    const int64_t chunk = 8192, rows = nt * P;
    const int NF = KSC_PRUNE_FEATURES, NP = KSC_PRUNE_NPARAMS;
    float *feats = nullptr, *lab = nullptr, *Y = nullptr, *dists = nullptr, *model = nullptr;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *xb = nullptr, *yb = nullptr, *lossd = nullptr;
    int32_t* probes = nullptr;
    int64_t *ids = nullptr, *idx = nullptr;
    int rc = KSC_OK;
    const int steps = (int)((rows + batch - 1) / batch);
    do {
        T_CUDA(cudaMalloc(&feats, sizeof(float) * rows * NF));
        T_CUDA(cudaMalloc(&lab, sizeof(float) * rows));
        T_CUDA(cudaMalloc(&Y, sizeof(float) * rows * 2));
        T_CUDA(cudaMalloc(&probes, sizeof(int32_t) * chunk * P));
        T_CUDA(cudaMalloc(&ids, sizeof(int64_t) * chunk * k));
        T_CUDA(cudaMalloc(&dists, sizeof(float) * chunk * k));
        T_CUDA(cudaMalloc(&model, sizeof(float) * KSC_PRUNE_MODEL));
        // 1. rows of the P nearest lists of every training query: labels from
        //    the plain search of those lists, features
        for (int64_t c0 = 0; c0 < nt && rc == KSC_OK; c0 += chunk) {
            const int64_t nc = std::min(chunk, nt - c0);
            const float* Qc = Qtrain_dev + c0 * rr_d(ix);
            const float* Qcw;
            if ((rc = work_queries(ix, Qc, nc, st, &Qcw))) break;
            if ((rc = rank_lists(ix, Qcw, nc, nullptr, P, P, probes, nullptr, RANK_TC16, st))) break;
            Plan pl;
            if ((rc = make_plan(ix, nc, k, P, R, nullptr, pl))) break;
            if ((rc = search_from_probes(ix, Qcw, pl, probes, ids, dists, nullptr, nullptr, st, Qc))) break;
            if ((rc = prune_labels(ix, ids, dists, nc, k, kth_dev + c0, probes, P, P, lab + c0 * P, st))) break;
            if ((rc = prune_rows(ix, Qcw, nc, probes, P, nullptr, P, 0.f, feats + c0 * P * NF, nullptr, nullptr,
                                 nullptr, st)))
                break;
        }
        if (rc) break;
        // 2. standardised features, targets
        if ((rc = prune_standardise(feats, rows, model, st))) break;
        if ((rc = prune_targets(lab, rows, Y, st))) break;
        // 3. weights: He-uniform from the seed, zero biases
        std::vector<float> wh(NP, 0.f);
        const int fan[3] = {NF, 32, 32}, nrow[3] = {32, 32, 2};
        int off = 0;
        for (int l = 0; l < 3; ++l) {
            const float a = sqrtf(6.f / fan[l]);
            for (int e = 0; e < nrow[l] * fan[l]; ++e)
                wh[off + e] = a * (2.f * (float)((mix64(seed) >> 11) * (1.0 / 9007199254740992.0)) - 1.f);
            off += nrow[l] * fan[l] + nrow[l];
        }
        T_CUDA(cudaMalloc(&w, sizeof(float) * NP));
        T_CUDA(cudaMalloc(&g, sizeof(float) * NP));
        T_CUDA(cudaMalloc(&m, sizeof(float) * NP));
        T_CUDA(cudaMalloc(&v, sizeof(float) * NP));
        T_CUDA(cudaMalloc(&xb, sizeof(float) * batch * NF));
        T_CUDA(cudaMalloc(&yb, sizeof(float) * batch * 2));
        T_CUDA(cudaMalloc(&idx, sizeof(int64_t) * rows));
        T_CUDA(cudaMalloc(&lossd, sizeof(float) * steps));
        T_CUDA(cudaMemcpy(w, wh.data(), sizeof(float) * NP, cudaMemcpyHostToDevice));
        T_CUDA(cudaMemset(m, 0, sizeof(float) * NP));
        T_CUDA(cudaMemset(v, 0, sizeof(float) * NP));
        // 4. Adam over shuffled minibatches of rows
        std::vector<int64_t> perm(rows);
        int t = 0;
        for (int ep = 0; ep < epochs && rc == KSC_OK; ++ep) {
            for (int64_t i = 0; i < rows; ++i) perm[i] = i;
            for (int64_t i = rows - 1; i > 0; --i) std::swap(perm[i], perm[(int64_t)(mix64(seed) % (uint64_t)(i + 1))]);
            T_CUDA(cudaMemcpyAsync(idx, perm.data(), sizeof(int64_t) * rows, cudaMemcpyHostToDevice, st));
            for (int s_ = 0; s_ < steps; ++s_) {
                const int64_t b0 = (int64_t)s_ * batch, nb = std::min<int64_t>(batch, rows - b0);
                k_gather_rows<<<(unsigned)((nb * NF + 255) / 256), 256, 0, st>>>(feats, idx + b0, nb, NF, xb);
                k_gather_rows<<<(unsigned)((nb * 2 + 255) / 256), 256, 0, st>>>(Y, idx + b0, nb, 2, yb);
                if ((rc = prune_mlp_grad(w, xb, yb, nb, g, lossd + s_, st))) break;
                if ((rc = mlp_adam_n(w, g, m, v, NP, ++t, lr, st))) break;
            }
            T_CUDA(cudaStreamSynchronize(st));  // perm is reused by the next epoch
        }
        if (rc) break;
        if (loss_host) {
            std::vector<float> lh(steps);
            T_CUDA(cudaMemcpy(lh.data(), lossd, sizeof(float) * steps, cudaMemcpyDeviceToHost));
            double sum = 0.0;
            for (float x : lh) sum += x;
            *loss_host = (float)(sum / steps);
        }
        T_CUDA(cudaMemcpy(model, w, sizeof(float) * NP, cudaMemcpyDeviceToDevice));
        if (ix->pr_model) cudaFree(ix->pr_model);
        ix->pr_model = model;
        model = nullptr;
        bump_workspace_generation();
    } while (0);
    void* tmp[] = {feats, lab, Y, dists, model, w, g, m, v, xb, yb, lossd, probes, ids, idx};
    for (void* p : tmp)
        if (p) cudaFree(p);
    return rc;
}
#undef T_CUDA

}  // extern "C"
