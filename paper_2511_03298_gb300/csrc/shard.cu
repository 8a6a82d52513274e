// List-sharded search: the inverted lists (and their vectors) partitioned over
// several index shards, one per GPU; centroids and codebooks replicated.
//
// Sec. 5.1 runs KScaNN as several processes (one per NUMA domain, throughput
// summed); for an index larger than one device the lists themselves are split.
// Every shard ranks all lists and builds the tables of every probed list from
// the replicated centroids and codebooks, so each computes the same per-query
// scale a_q (Sec. 2.5 quantisation over the whole probe set) and its keys are
// comparable with every other shard's.  Per search:
//   1. ksc_shard_candidates: steps a1 .. a5 on the shard's own lists -> its R
//      smallest keys, global ids (rows are kept in ascending global id, so the
//      local order of (distance, id) is the global one);
//   2. exchange: every shard receives all shards' keys (an all-gather);
//   3. ksc_shard_rerank: theta = the R-th smallest key of all of them (the
//      whole index's R-th key); the shard re-ranks exactly its own keys at or
//      below theta (its members of the global top R) -> its k best;
//   4. exchange of the (distance, id) lists, then ksc_merge_topk.
// The union of the shards' candidates at or below theta is exactly the
// unsharded search's candidate set, and each is re-ranked by the same kernel
// on the same row, so the merged result equals the unsharded one.
#include <algorithm>

#include "index.cuh"

namespace ksc {

constexpr int SH_MAX_KEYS = 8192;  // keys a CTA sorts in shared memory

// Low word of every real key: local row -> global id.
__global__ void k_keys_to_global(uint64_t* __restrict__ keys, int64_t n, const int32_t* __restrict__ gids) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        if (k != KEY_NONE) keys[i] = (k & 0xffffffff00000000ull) | (uint32_t)gids[(uint32_t)k];
    }
}

// First local row whose global id is >= g (gids ascending).
__device__ __forceinline__ int32_t local_row(const int32_t* __restrict__ gids, int64_t n, int32_t g) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (gids[mid] < g) lo = mid + 1;
        else hi = mid;
    }
    return (int32_t)lo;
}

// Per query (one CTA): theta = the R-th smallest of the parts x R gathered
// keys (all[part][q][j], KEY_NONE pads, sorted in shared memory), then the
// shard's own keys (own[q][j], global ids) at or below theta, as local-row
// keys into out[q][j] (KEY_NONE elsewhere).
__global__ void __launch_bounds__(256) k_shard_select(const uint64_t* __restrict__ all, int parts, int64_t nq, int R,
                                                      const uint64_t* __restrict__ own,
                                                      const int32_t* __restrict__ gids, int64_t n_local,
                                                      uint64_t* __restrict__ out) {
    extern __shared__ uint64_t sk[];
    __shared__ unsigned long long s_theta;
    const int64_t q = blockIdx.x;
    const int W = parts * R, S = pow2_ceil(W < 2 ? 2 : W);
    for (int i = threadIdx.x; i < S; i += blockDim.x) {
        const int g = i / R, j = i - g * R;
        sk[i] = i < W ? all[((int64_t)g * nq + q) * R + j] : KEY_NONE;
    }
    __syncthreads();
    block_bitonic_sort(sk, S);
    if (threadIdx.x == 0) s_theta = sk[R - 1];
    __syncthreads();
    const uint64_t theta = s_theta;
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        const uint64_t k = own[q * R + j];
        uint64_t o = KEY_NONE;
        if (k != KEY_NONE && k <= theta) {
            const int32_t r = local_row(gids, n_local, (int32_t)(uint32_t)k);
            o = (k & 0xffffffff00000000ull) | (uint32_t)r;
        }
        out[q * R + j] = o;
    }
}

__global__ void k_ids_to_global(int64_t* __restrict__ ids, int64_t n, const int32_t* __restrict__ gids) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (ids[i] >= 0) ids[i] = gids[ids[i]];
}

// Final merge (one CTA per query): the k best of parts x k (distance, id)
// pairs (ids[part][q][i], dists[part][q][i]) by distance (ascending for L2,
// similarity descending for inner product), then id; pads (id -1) last.
__global__ void __launch_bounds__(256) k_merge_topk(const int64_t* __restrict__ ids, const float* __restrict__ dists,
                                                    int64_t nq, int parts, int k, int ip,
                                                    int64_t* __restrict__ out_ids, float* __restrict__ out_d) {
    extern __shared__ uint64_t sm[];
    const int64_t q = blockIdx.x;
    const int W = parts * k, S = pow2_ceil(W < 2 ? 2 : W);
    for (int i = threadIdx.x; i < S; i += blockDim.x) {
        uint64_t key = KEY_NONE;
        if (i < W) {
            const int g = i / k, j = i - g * k;
            const int64_t at = ((int64_t)g * nq + q) * k + j;
            const int64_t id = ids[at];
            const float v = ip ? -dists[at] : dists[at];
            key = id < 0 ? KEY_NONE : (((uint64_t)ordered_f32(v) << 32) | (uint32_t)id);
        }
        sm[i] = key;
    }
    __syncthreads();
    block_bitonic_sort(sm, S);
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const uint64_t key = sm[i];
        if (key == KEY_NONE) {
            out_ids[q * k + i] = -1;
            out_d[q * k + i] = ip ? -INFINITY : INFINITY;
        } else {
            const float v = unordered_f32((uint32_t)(key >> 32));
            out_ids[q * k + i] = (int64_t)(uint32_t)key;
            out_d[q * k + i] = ip ? -v : v;
        }
    }
}

static unsigned grid_of(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4096); }

}  // namespace ksc

using namespace ksc;

extern "C" {

int ksc_shard_candidates(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t nprobe, int32_t rerank, int32_t k,
                         uint64_t* keys_dev, const ksc_search_opts* opts, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    KSC_CHECK_ARG(ix->gids, "not a shard (see ksc_index_import_shard)");
    KSC_CHECK_ARG(k >= 1 && k <= KSC_MAX_K, "k must be in [1, %d]", KSC_MAX_K);
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && keys_dev, "null argument");
    const int R = std::max(rerank, k);
    cudaStream_t st = as_stream(stream);
    KSC_TRY(search_keys(ix, Q_dev, nq, nprobe, R, opts, keys_dev, st));
    k_keys_to_global<<<grid_of(nq * R), 256, 0, st>>>(keys_dev, nq * R, ix->gids);
    KSC_LAUNCH_CHECK();
    ix->launches++;
    return KSC_OK;
}

int ksc_shard_rerank(ksc_index* ix, const float* Q_dev, int64_t nq, int32_t k, int32_t rerank,
                     const uint64_t* own_keys_dev, const uint64_t* all_keys_dev, int32_t parts, int64_t* ids_dev,
                     float* dists_dev, void* stream) {
    KSC_CHECK_ARG(ix, "null index");
    KSC_CHECK_ARG(ix->gids, "not a shard (see ksc_index_import_shard)");
    KSC_CHECK_ARG(k >= 1 && k <= KSC_MAX_K, "k must be in [1, %d]", KSC_MAX_K);
    const int R = std::max(rerank, k);
    KSC_CHECK_ARG(R <= KSC_MAX_RERANK, "rerank must be <= %d", KSC_MAX_RERANK);
    KSC_CHECK_ARG(parts >= 1 && (int64_t)parts * R <= SH_MAX_KEYS, "parts x R must be in [1, %d]", SH_MAX_KEYS);
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(Q_dev && own_keys_dev && all_keys_dev && ids_dev && dists_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    KSC_TRY(ensure(ix->ws_topr2, sizeof(uint64_t) * nq * R, st));
    uint64_t* mine = (uint64_t*)ix->ws_topr2.p;
    const size_t smem = sizeof(uint64_t) * pow2_ceil(parts * R < 2 ? 2 : parts * R);
    KSC_CUDA(cudaFuncSetAttribute(k_shard_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_shard_select<<<(unsigned)nq, 256, smem, st>>>(all_keys_dev, parts, nq, R, own_keys_dev, ix->gids, ix->n, mine);
    KSC_LAUNCH_CHECK();
    KSC_TRY(rerank_keys(ix, Q_dev, nq, k, mine, R, ids_dev, dists_dev, st));
    k_ids_to_global<<<grid_of(nq * k), 256, 0, st>>>(ids_dev, nq * k, ix->gids);
    KSC_LAUNCH_CHECK();
    ix->launches += 2;
    return KSC_OK;
}

int ksc_merge_topk(const int64_t* ids_dev, const float* dists_dev, int64_t nq, int32_t parts, int32_t k,
                   int32_t ip, int64_t* ids_out_dev, float* dists_out_dev, void* stream) {
    KSC_CHECK_ARG(k >= 1 && k <= KSC_MAX_K, "k must be in [1, %d]", KSC_MAX_K);
    KSC_CHECK_ARG(parts >= 1 && (int64_t)parts * k <= SH_MAX_KEYS, "parts x k must be in [1, %d]", SH_MAX_KEYS);
    KSC_CHECK_ARG(nq >= 0, "nq < 0");
    if (nq == 0) return KSC_OK;
    KSC_CHECK_ARG(ids_dev && dists_dev && ids_out_dev && dists_out_dev, "null argument");
    cudaStream_t st = as_stream(stream);
    const size_t smem = sizeof(uint64_t) * pow2_ceil(parts * k < 2 ? 2 : parts * k);
    KSC_CUDA(cudaFuncSetAttribute(k_merge_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_merge_topk<<<(unsigned)nq, 256, smem, st>>>(ids_dev, dists_dev, nq, parts, k, ip != 0, ids_out_dev,
                                                 dists_out_dev);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

}  // extern "C"
