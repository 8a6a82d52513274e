// Intra-list graphs for the hybrid search (Sec. 4.4, Alg. 1 BuildGraph).
//
// Graph: for every vector, its 32 nearest other members of the same list
// (exact FP32 squared distance on the stored vectors, ties -> lower id;
// lists with fewer members are padded with -1).  Entry of a list: the member
// nearest its mean centroid.  For the search the graph is re-expressed per
// list position, and every node carries a copy of its 32 neighbours' codes in
// the block layout, so one node expansion is one LUT16 block (the paper's
// 32-point adjacency blocks).
#include <vector>

#include "index.cuh"

namespace ksc {

__device__ __forceinline__ uint64_t dkey(float d, int32_t id) {
    return ((uint64_t)ordered_f32(d) << 32) | (uint32_t)id;
}

// Warp-wide bitonic sort of one key per lane, ascending across lanes.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool up = (lane & k) == 0;
            const bool lower = (lane & j) == 0;
            // keep the smaller in the lower lane of an ascending pair
            v = (lower == up) ? (v < o ? v : o) : (v < o ? o : v);
        }
    }
    return v;
}

// top (ascending, lane l = l-th smallest) merged with a sorted chunk: the 32
// smallest of both, ascending.
__device__ __forceinline__ uint64_t warp_merge32(uint64_t top, uint64_t chunk_sorted, int lane) {
    // pair top[l] with chunk[31 - l]: the minima form a bitonic sequence
    const uint64_t rev = __shfl_sync(0xffffffffu, chunk_sorted, 31 - lane);
    uint64_t v = top < rev ? top : rev;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
        const bool lower = (lane & j) == 0;
        v = lower ? (v < o ? v : o) : (v < o ? o : v);
    }
    return v;
}

// One CTA per 32-vector block of a list: distances from its 32 members to
// every member of the list, tiled 32 x 32 through shared memory, and a
// running top-32 per member kept one key per lane.
constexpr int KG_D = 128;  // dimensions staged per pass
__global__ void __launch_bounds__(256) k_knn_graph(const float* __restrict__ X, int d, const int32_t* __restrict__ blk_ids,
                                                   const int32_t* __restrict__ blk_list,
                                                   const int64_t* __restrict__ boff, int32_t* __restrict__ graph) {
    __shared__ float xu[32][KG_D + 1];
    __shared__ float xv[32][KG_D + 1];
    __shared__ float dist[32][33];
    const int64_t b = blockIdx.x;
    const int p = blk_list[b];
    const int64_t s0 = boff[p] * 32, s1 = boff[p + 1] * 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t uid = blk_ids[b * 32 + lane];  // same in every warp
    uint64_t top[4];                             // warp w keeps members u = 4w .. 4w+3
#pragma unroll
    for (int i = 0; i < 4; ++i) top[i] = KEY_NONE;
    for (int64_t t0 = s0; t0 < s1; t0 += 32) {
        const int32_t vid = blk_ids[t0 + lane];
        // 32 x 32 squared distances, d in passes of KG_D
        float acc[4] = {0.f, 0.f, 0.f, 0.f};  // thread: u = threadIdx.x / 8 .. (4 pairs)
        for (int k0 = 0; k0 < d; k0 += KG_D) {
            const int kd = min(KG_D, d - k0);
            __syncthreads();
            for (int e = threadIdx.x; e < 32 * KG_D; e += blockDim.x) {
                const int r = e / KG_D, c = e - r * KG_D;
                const int32_t iu = blk_ids[b * 32 + r], iv = blk_ids[t0 + r];
                xu[r][c] = (c < kd && iu >= 0) ? X[(int64_t)iu * d + k0 + c] : 0.f;
                xv[r][c] = (c < kd && iv >= 0) ? X[(int64_t)iv * d + k0 + c] : 0.f;
            }
            __syncthreads();
            const int ui = threadIdx.x >> 3, vj = (threadIdx.x & 7) * 4;
            for (int c = 0; c < kd; ++c) {
                const float a = xu[ui][c];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float e = a - xv[vj + q][c];
                    acc[q] = fmaf(e, e, acc[q]);
                }
            }
        }
        {
            const int ui = threadIdx.x >> 3, vj = (threadIdx.x & 7) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) dist[ui][vj + q] = acc[q];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int u = w * 4 + i;
            const int32_t me = __shfl_sync(0xffffffffu, uid, u);
            uint64_t k = (vid >= 0 && vid != me && me >= 0) ? dkey(dist[u][lane], vid) : KEY_NONE;
            k = warp_sort32(k, lane);
            top[i] = warp_merge32(top[i], k, lane);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int u = w * 4 + i;
        const int32_t me = __shfl_sync(0xffffffffu, uid, u);
        if (me >= 0) graph[(int64_t)me * 32 + lane] = top[i] == KEY_NONE ? -1 : (int32_t)(top[i] & 0xffffffffu);
    }
}

// Entry of every list: the member nearest its mean centroid (ties -> lower id).
__global__ void k_graph_entry(const float* __restrict__ X, int d, const float* __restrict__ c_mean,
                              const int32_t* __restrict__ blk_ids, const int64_t* __restrict__ boff, int L,
                              int32_t* __restrict__ entry) {
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= L) return;
    uint64_t best = KEY_NONE;
    for (int64_t s = boff[p] * 32 + lane; s < boff[p + 1] * 32; s += 32) {
        const int32_t id = blk_ids[s];
        if (id < 0) continue;
        float acc = 0.f;
        for (int t = 0; t < d; ++t) {
            const float e = X[(int64_t)id * d + t] - c_mean[(int64_t)p * d + t];
            acc = fmaf(e, e, acc);
        }
        const uint64_t k = dkey(acc, id);
        best = k < best ? k : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t x = __shfl_xor_sync(0xffffffffu, best, o);
        best = x < best ? x : best;
    }
    if (lane == 0) entry[p] = best == KEY_NONE ? -1 : (int32_t)(best & 0xffffffffu);
}

// Position of every vector inside its list (slot - first slot of the list).
__global__ void k_positions(const int32_t* __restrict__ blk_ids, const int32_t* __restrict__ blk_list,
                            const int64_t* __restrict__ boff, int64_t nslots, int32_t* __restrict__ pos_of) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    const int32_t id = blk_ids[s];
    if (id >= 0) pos_of[id] = (int32_t)(s - boff[blk_list[s >> 5]] * 32);
}

// Per slot: the 32 neighbours as list positions, and their codes as one block.
__global__ void k_graph_prepare(const int32_t* __restrict__ graph, const int32_t* __restrict__ pos_of,
                                const int32_t* __restrict__ blk_ids, const int32_t* __restrict__ blk_list,
                                const int64_t* __restrict__ boff, const uint8_t* __restrict__ blk_codes, int M,
                                int64_t nslots, int32_t* __restrict__ nbr_pos, uint8_t* __restrict__ nbr_codes) {
    const int64_t tot = nslots * M * 16;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e & 15);
        const int64_t sj = e >> 4;
        const int j = (int)(sj % M);
        const int64_t s = sj / M;
        const int32_t u = blk_ids[s];
        const int64_t base = boff[blk_list[s >> 5]] * 32;
        uint32_t byte = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nb = 2 * i + h;
            const int32_t v = u >= 0 ? graph[(int64_t)u * 32 + nb] : -1;
            if (v >= 0) {
                const int64_t sv = base + pos_of[v];
                const uint8_t cb = blk_codes[((sv >> 5) * M + j) * 16 + ((sv & 31) >> 1)];
                byte |= (uint32_t)((sv & 1) ? (cb >> 4) : (cb & 15)) << (4 * h);
            }
            if (j == 0 && i < 16) nbr_pos[s * 32 + nb] = v >= 0 ? pos_of[v] : -1;
        }
        nbr_codes[e] = (uint8_t)byte;
    }
}

static int grid_for_g(int64_t work) {
    int64_t g = (work + 255) / 256;
    int64_t cap = (int64_t)num_sms() * 16;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// From graph / entry in global ids (already on the device): the search form.
int prepare_graph(ksc_index* ix, cudaStream_t st) {
    const int64_t nslots = ix->nblocks * 32;
    int32_t* pos_of = nullptr;
    KSC_CUDA(cudaMalloc(&pos_of, sizeof(int32_t) * ix->n));
    k_positions<<<(unsigned)((nslots + 255) / 256), 256, 0, st>>>(ix->blk_ids, ix->blk_list, ix->list_boff, nslots,
                                                                  pos_of);
    if (ix->nbr_pos) cudaFree(ix->nbr_pos);
    if (ix->nbr_codes) cudaFree(ix->nbr_codes);
    if (ix->entry_pos) cudaFree(ix->entry_pos);
    cudaError_t e1 = cudaMalloc(&ix->nbr_pos, sizeof(int32_t) * nslots * 32);
    cudaError_t e2 = cudaMalloc(&ix->nbr_codes, (size_t)nslots * ix->M * 16);
    cudaError_t e3 = cudaMalloc(&ix->entry_pos, sizeof(int32_t) * ix->L);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        cudaFree(pos_of);
        set_error("graph allocation failed");
        return KSC_ENOMEM;
    }
    k_graph_prepare<<<grid_for_g(nslots * ix->M * 16), 256, 0, st>>>(ix->graph, pos_of, ix->blk_ids, ix->blk_list,
                                                                     ix->list_boff, ix->blk_codes, ix->M, nslots,
                                                                     ix->nbr_pos, ix->nbr_codes);
    // entry positions (host: L values)
    std::vector<int32_t> ent(ix->L), pos(ix->n);
    KSC_CUDA(cudaMemcpyAsync(ent.data(), ix->entry, sizeof(int32_t) * ix->L, cudaMemcpyDeviceToHost, st));
    KSC_CUDA(cudaMemcpyAsync(pos.data(), pos_of, sizeof(int32_t) * ix->n, cudaMemcpyDeviceToHost, st));
    KSC_CUDA(cudaStreamSynchronize(st));
    for (int p = 0; p < ix->L; ++p) ent[p] = ent[p] >= 0 ? pos[ent[p]] : -1;
    KSC_CUDA(cudaMemcpy(ix->entry_pos, ent.data(), sizeof(int32_t) * ix->L, cudaMemcpyHostToDevice));
    cudaFree(pos_of);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

int build_graph(ksc_index* ix, cudaStream_t st) {
    if (!ix->graph) KSC_CUDA(cudaMalloc(&ix->graph, sizeof(int32_t) * ix->n * 32));
    if (!ix->entry) KSC_CUDA(cudaMalloc(&ix->entry, sizeof(int32_t) * ix->L));
    k_knn_graph<<<(unsigned)ix->nblocks, 256, 0, st>>>(ix->X, ix->d, ix->blk_ids, ix->blk_list, ix->list_boff,
                                                      ix->graph);
    KSC_LAUNCH_CHECK();
    k_graph_entry<<<(ix->L + 7) / 8, 256, 0, st>>>(ix->X, ix->d, ix->c_mean, ix->blk_ids, ix->list_boff, ix->L,
                                                    ix->entry);
    KSC_LAUNCH_CHECK();
    return prepare_graph(ix, st);
}

}  // namespace ksc
