// Index construction (Alg. 1), import / export and memory management.
//
// build: IVF k-means (Lloyd, Sec. 2.2) on a sample, list assignment by the
// ranking score, mean centroids for residuals (Sec. 4.6.1), PQ codebooks with
// K = 16 per subspace on residuals (Sec. 2.3), encoding, block packing
// (Alg. 1 BuildBlocks).  All on the GPU in FP32 (sums in FP64); the list
// ordering (a counting sort of the assignment) runs on the host.
#include <atomic>
#include <cstdarg>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "index.cuh"

namespace ksc {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char* get_error() { return g_err; }

static std::atomic<unsigned long long> g_ws_gen{0};
unsigned long long workspace_generation() { return g_ws_gen.load(); }
void bump_workspace_generation() { g_ws_gen++; }

int ensure(Buffer& b, size_t bytes, cudaStream_t st) {
    if (bytes <= b.bytes && b.p) return KSC_OK;
    g_ws_gen++;
    if (b.p) {
        KSC_CUDA(cudaStreamSynchronize(st));
        KSC_CUDA(cudaFree(b.p));
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = bytes < 256 ? 256 : bytes;
    want = (want + 255) & ~size_t(255);
    KSC_CUDA(cudaMalloc(&b.p, want));
    b.bytes = want;
    return KSC_OK;
}

void release(Buffer& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// ------------------------------------------------------------------ kernels
__global__ void k_gather_rows(const float* __restrict__ X, const int64_t* __restrict__ idx, int64_t cnt,
                              int d, float* __restrict__ out) {
    int64_t tot = cnt * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / d;
        int t = (int)(e - r * d);
        out[e] = X[idx[r] * d + t];
    }
}

__global__ void k_row_sqnorm(const float* __restrict__ C, int L, int d, float* __restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L) return;
    float s = 0.f;
    for (int t = 0; t < d; ++t) s = fmaf(C[(int64_t)c * d + t], C[(int64_t)c * d + t], s);
    out[c] = s;
}

__global__ void k_normalise_rows(float* __restrict__ C, int L, int d) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L) return;
    double s = 0.0;
    for (int t = 0; t < d; ++t) s += (double)C[(int64_t)c * d + t] * C[(int64_t)c * d + t];
    if (s > 0.0) {
        double inv = 1.0 / sqrt(s);
        for (int t = 0; t < d; ++t) C[(int64_t)c * d + t] = (float)(C[(int64_t)c * d + t] * inv);
    }
}

// Nearest centroid of every row: score = ||c||^2 - 2<x,c> (L2) or -<x,c>
// (spherical); ties -> lower centroid id.  64 rows x 64 centroids per tile,
// 256 threads, 4 x 4 outputs per thread, dims staged 32 at a time.
constexpr int AS_T = 64, AS_K = 32;
__global__ void __launch_bounds__(256) k_assign(const float* __restrict__ X, int64_t np, int d,
                                                const float* __restrict__ Cc, const float* __restrict__ cn,
                                                int L, int spherical, int32_t* __restrict__ assign,
                                                float* __restrict__ best_out) {
    __shared__ float xs[AS_K][AS_T + 4];
    __shared__ float cs[AS_K][AS_T + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * AS_T;
    float best[4];
    int bid[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { best[i] = INFINITY; bid[i] = 0x7fffffff; }
    for (int c0 = 0; c0 < L; c0 += AS_T) {
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int k0 = 0; k0 < d; k0 += AS_K) {
            for (int e = threadIdx.x; e < AS_T * AS_K; e += 256) {
                int r = e / AS_K, kk = e % AS_K;
                int64_t gr = row0 + r;
                int gk = k0 + kk;
                xs[kk][r] = (gr < np && gk < d) ? X[gr * d + gk] : 0.f;
                int gc = c0 + r;
                cs[kk][r] = (gc < L && gk < d) ? Cc[(int64_t)gc * d + gk] : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < AS_K; ++kk) {
                float a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = xs[kk][ty * 4 + i];
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
        for (int j = 0; j < 4; ++j) {
            int c = c0 + tx * 4 + j;
            if (c >= L) continue;
            float base = spherical ? 0.f : cn[c];
            float mul = spherical ? -1.f : -2.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float s = fmaf(mul, acc[i][j], base);
                if (s < best[i] || (s == best[i] && c < bid[i])) { best[i] = s; bid[i] = c; }
            }
        }
    }
    // reduce over the 16 threads (tx) that share these rows
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float ob = __shfl_xor_sync(0xffffffffu, best[i], off);
            int oi = __shfl_xor_sync(0xffffffffu, bid[i], off);
            if (ob < best[i] || (ob == best[i] && oi < bid[i])) { best[i] = ob; bid[i] = oi; }
        }
    }
    if (tx == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int64_t r = row0 + ty * 4 + i;
            if (r < np) {
                assign[r] = bid[i];
                if (best_out) best_out[r] = best[i];
            }
        }
    }
}

// Accumulate rows into per-centroid FP64 sums (X rows, optional row index map).
__global__ void k_centroid_accum(const float* __restrict__ X, const int64_t* __restrict__ idx, int64_t np,
                                 int d, const int32_t* __restrict__ a, double* __restrict__ sums,
                                 unsigned long long* __restrict__ cnt) {
    int64_t tot = np * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / d;
        int t = (int)(e - r * d);
        int64_t src = idx ? idx[r] : r;
        int c = a[r];
        atomicAdd(&sums[(int64_t)c * d + t], (double)X[src * d + t]);
        if (t == 0) atomicAdd(&cnt[c], 1ull);
    }
}

__global__ void k_centroid_finish(const double* __restrict__ sums, const unsigned long long* __restrict__ cnt,
                                  const float* __restrict__ fallback, int L, int d, float* __restrict__ out) {
    int64_t tot = (int64_t)L * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(e / d);
        out[e] = cnt[c] > 0 ? (float)(sums[e] / (double)cnt[c]) : fallback[e];
    }
}

// residual rows r = x - c_mean[a(x)] (one fp32 subtraction)
__global__ void k_residual(const float* __restrict__ X, const int64_t* __restrict__ idx, int64_t cnt, int d,
                           const int32_t* __restrict__ assign, const float* __restrict__ c_mean,
                           float* __restrict__ out) {
    int64_t tot = cnt * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / d;
        int t = (int)(e - r * d);
        int64_t src = idx ? idx[r] : r;
        out[e] = __fsub_rn(X[src * d + t], c_mean[(int64_t)assign[src] * d + t]);
    }
}

// PQ: nearest of the 16 codewords of subspace j for residual rows (one
// thread per (row, j)); rows either given as residuals R or computed from X.
__global__ void k_pq_encode(const float* __restrict__ R, const float* __restrict__ X,
                            const int32_t* __restrict__ assign, const float* __restrict__ c_mean, int64_t np,
                            int d, int M, int dsub, const float* __restrict__ cb, uint8_t* __restrict__ codes) {
    int64_t tot = np * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / M;
        int j = (int)(e - r * M);
        float best = INFINITY;
        int bi = 0;
        for (int c = 0; c < PQ_K; ++c) {
            const float* w = cb + ((int64_t)j * PQ_K + c) * dsub;
            float s = 0.f;
            for (int t = 0; t < dsub; ++t) {
                int tt = j * dsub + t;
                float rv = R ? R[r * d + tt] : __fsub_rn(X[r * d + tt], c_mean[(int64_t)assign[r] * d + tt]);
                float df = rv - w[t];
                s = fmaf(df, df, s);
            }
            if (s < best) { best = s; bi = c; }
        }
        codes[e] = (uint8_t)bi;
    }
}

__global__ void k_pq_accum(const float* __restrict__ R, int64_t np, int d, int M, int dsub,
                           const uint8_t* __restrict__ codes, double* __restrict__ sums,
                           unsigned long long* __restrict__ cnt) {
    int64_t tot = np * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / d;
        int tt = (int)(e - r * d);
        int j = tt / dsub, t = tt - j * dsub;
        int c = codes[r * M + j];
        atomicAdd(&sums[((int64_t)j * PQ_K + c) * dsub + t], (double)R[e]);
        if (t == 0) atomicAdd(&cnt[(int64_t)j * PQ_K + c], 1ull);
    }
}

__global__ void k_pq_finish(const double* __restrict__ sums, const unsigned long long* __restrict__ cnt, int M,
                            int dsub, float* __restrict__ cb) {
    int64_t tot = (int64_t)M * PQ_K * dsub;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t jc = e / dsub;
        if (cnt[jc] > 0) cb[e] = (float)(sums[e] / (double)cnt[jc]);
    }
}

__global__ void k_pq_init(const float* __restrict__ R, int d, int M, int dsub, float* __restrict__ cb) {
    // codeword c of subspace j = sub-vector j of sample row c
    int64_t tot = (int64_t)M * PQ_K * dsub;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int t = (int)(e % dsub);
        int64_t jc = e / dsub;
        int c = (int)(jc % PQ_K), j = (int)(jc / PQ_K);
        cb[e] = R[(int64_t)c * d + j * dsub + t];
    }
}

// Pack unpacked codes [n x M] into the block layout given the block member ids.
__global__ void k_pack(const int32_t* __restrict__ blk_ids, int64_t nblocks, int M,
                       const uint8_t* __restrict__ codes, uint8_t* __restrict__ blk_codes) {
    int64_t tot = nblocks * M * 16;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e & 15);
        int64_t bj = e >> 4;
        int j = (int)(bj % M);
        int64_t b = bj / M;
        int32_t id0 = blk_ids[b * 32 + 2 * i], id1 = blk_ids[b * 32 + 2 * i + 1];
        uint32_t lo = id0 >= 0 ? codes[(int64_t)id0 * M + j] : 0u;
        uint32_t hi = id1 >= 0 ? codes[(int64_t)id1 * M + j] : 0u;
        blk_codes[e] = (uint8_t)(lo | (hi << 4));
    }
}

// Unpack the block layout back to codes [n x M].
__global__ void k_unpack(const int32_t* __restrict__ blk_ids, int64_t nblocks, int M,
                         const uint8_t* __restrict__ blk_codes, uint8_t* __restrict__ codes) {
    int64_t tot = nblocks * 32 * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(e % M);
        int64_t bv = e / M;
        int v = (int)(bv & 31);
        int64_t b = bv >> 5;
        int32_t id = blk_ids[b * 32 + v];
        if (id < 0) continue;
        uint8_t byte = blk_codes[(b * M + j) * 16 + (v >> 1)];
        codes[(int64_t)id * M + j] = (v & 1) ? (byte >> 4) : (byte & 15);
    }
}

static int grid_for(int64_t work, int threads = 256) {
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// ------------------------------------------------------------------ host helpers
static int alloc_copy(void** dst, const void* src, size_t bytes, cudaStream_t st, cudaMemcpyKind kind) {
    KSC_CUDA(cudaMalloc(dst, bytes < 16 ? 16 : bytes));
    if (src && bytes) KSC_CUDA(cudaMemcpyAsync(*dst, src, bytes, kind, st));
    return KSC_OK;
}

// The search workspace buffers of a handle.
static int workspace_buffers(ksc_index* ix, Buffer** out) {
    Buffer* bufs[] = {&ix->ws_scores, &ix->ws_probes, &ix->ws_lut, &ix->ws_bias, &ix->ws_scale, &ix->ws_range,
                      &ix->ws_thr, &ix->ws_cnt, &ix->ws_cand, &ix->ws_topr, &ix->ws_nprobe, &ix->ws_rerank,
                      &ix->ws_items, &ix->ws_misc, &ix->ws_qbf16, &ix->ws_err, &ix->ws_feat, &ix->ws_rscore,
                      &ix->ws_full, &ix->ws_topr2, &ix->ws_flag, &ix->ws_redo, &ix->ws_pprobes, &ix->ws_pn, &ix->ws_pprob, &ix->ws_qf};
    const int n = (int)(sizeof(bufs) / sizeof(bufs[0]));
    for (int i = 0; i < n; ++i) out[i] = bufs[i];
    return n;
}

int free_index_memory(ksc_index* ix) {
    Buffer* bufs[64];
    const int nb = workspace_buffers(ix, bufs);
    if (ix->parent) {
        // a view: its own workspace, status, counters and events, and what it
        // allocated lazily itself (not the same pointer as its source's)
        const ksc_index* s = ix->parent;
        void* own[] = {ix->status, ix->stats, ix->c_rank_bf16 != s->c_rank_bf16 ? ix->c_rank_bf16 : nullptr,
                       ix->c_rank_f8 != s->c_rank_f8 ? ix->c_rank_f8 : nullptr,
                       ix->c_rank_f8_scale != s->c_rank_f8_scale ? ix->c_rank_f8_scale : nullptr,
                       ix->X_bf16 != s->X_bf16 ? ix->X_bf16 : nullptr, ix->X_fp8 != s->X_fp8 ? ix->X_fp8 : nullptr,
                       ix->X_scale != s->X_scale ? ix->X_scale : nullptr,
                       ix->X_band != s->X_band ? ix->X_band : nullptr,
                       ix->X_u8 != s->X_u8 ? ix->X_u8 : nullptr};
        for (void* p : own)
            if (p) cudaFree(p);
        for (int i = 0; i < nb; ++i) release(*bufs[i]);
        for (int i = 0; i <= KSC_NUM_STAGES; ++i)
            if (ix->ev[i]) cudaEventDestroy(ix->ev[i]);
        return KSC_OK;
    }
    void* ptrs[] = {ix->X, ix->c_rank, ix->c_rank_sq, ix->c_mean, ix->codebook, ix->list_boff, ix->list_n,
                    ix->blk_ids, ix->blk_codes, ix->assign, ix->graph, ix->entry, ix->status, ix->stats,
                    ix->c_rank_bf16, ix->mlp_w, ix->blk_list, ix->nbr_pos, ix->nbr_codes, ix->entry_pos,
                    ix->X_bf16, ix->X_fp8, ix->X_scale, ix->pr_stats, ix->pr_vecs, ix->pr_model, ix->dims,
                    ix->X_rr, ix->c_rank_f8, ix->c_rank_f8_scale, ix->gids, ix->X_band, ix->X_u8};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < nb; ++i) release(*bufs[i]);
    for (int i = 0; i <= KSC_NUM_STAGES; ++i)
        if (ix->ev[i]) cudaEventDestroy(ix->ev[i]);
    return KSC_OK;
}

int pack_lists(ksc_index* ix, const uint8_t* codes_dev, const int32_t* assign_host, cudaStream_t st) {
    const int L = ix->L;
    const int64_t n = ix->n;
    std::vector<int64_t> cnt(L, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (assign_host[i] < 0 || assign_host[i] >= L) {
            set_error("assignment of row %lld out of range", (long long)i);
            return KSC_EINVAL;
        }
        cnt[assign_host[i]]++;
    }
    ix->h_boff.assign(L + 1, 0);
    ix->h_n.assign(L, 0);
    int64_t maxl = 0;
    for (int c = 0; c < L; ++c) {
        ix->h_n[c] = (int32_t)cnt[c];
        ix->h_boff[c + 1] = ix->h_boff[c] + (cnt[c] + BLOCK_VECS - 1) / BLOCK_VECS;
        if (cnt[c] > maxl) maxl = cnt[c];
    }
    ix->max_list = (int32_t)maxl;
    ix->nblocks = ix->h_boff[L];
    std::vector<int32_t> ids((size_t)ix->nblocks * BLOCK_VECS, -1);
    std::vector<int64_t> fill(L);
    for (int c = 0; c < L; ++c) fill[c] = ix->h_boff[c] * BLOCK_VECS;
    for (int64_t i = 0; i < n; ++i) ids[fill[assign_host[i]]++] = (int32_t)i;  // ascending id per list
    std::vector<int32_t> blist(ix->nblocks);
    for (int c = 0; c < L; ++c)
        for (int64_t bb = ix->h_boff[c]; bb < ix->h_boff[c + 1]; ++bb) blist[bb] = c;
    KSC_TRY(alloc_copy((void**)&ix->blk_list, blist.data(), sizeof(int32_t) * (ix->nblocks > 0 ? ix->nblocks : 1), st,
                       cudaMemcpyHostToDevice));
    KSC_TRY(alloc_copy((void**)&ix->list_boff, ix->h_boff.data(), sizeof(int64_t) * (L + 1), st, cudaMemcpyHostToDevice));
    KSC_TRY(alloc_copy((void**)&ix->list_n, ix->h_n.data(), sizeof(int32_t) * L, st, cudaMemcpyHostToDevice));
    KSC_TRY(alloc_copy((void**)&ix->blk_ids, ids.data(), sizeof(int32_t) * ids.size(), st, cudaMemcpyHostToDevice));
    KSC_CUDA(cudaMalloc(&ix->blk_codes, (size_t)ix->nblocks * ix->M * 16 + 16));
    k_pack<<<grid_for(ix->nblocks * ix->M * 16), 256, 0, st>>>(ix->blk_ids, ix->nblocks, ix->M, codes_dev,
                                                               ix->blk_codes);
    KSC_LAUNCH_CHECK();
    KSC_CUDA(cudaStreamSynchronize(st));  // `ids` goes out of scope
    return KSC_OK;
}

// splitmix64 (Steele, Lea, Flood 2014) driving a Fisher-Yates shuffle.
static uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void host_perm(int64_t n, uint64_t seed, std::vector<int64_t>& p) {
    p.resize(n);
    for (int64_t i = 0; i < n; ++i) p[i] = i;
    uint64_t s = seed;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)(splitmix64(s) % (uint64_t)(i + 1));
        int64_t t = p[i];
        p[i] = p[j];
        p[j] = t;
    }
}

// Lloyd on rows `sample` of X (device), init = first L sample rows.
static int lloyd(const float* X, const int64_t* sample_dev, int64_t ns, int d, int L, int iters, float* C,
                 cudaStream_t st) {
    float* Xs = nullptr;
    float* cn = nullptr;
    int32_t* a = nullptr;
    double* sums = nullptr;
    unsigned long long* cnt = nullptr;
    int rc = KSC_OK;
    auto cleanup = [&]() {
        cudaFree(Xs); cudaFree(cn); cudaFree(a); cudaFree(sums); cudaFree(cnt);
    };
#define LL_CUDA(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { set_error("%s: %s", #call, cudaGetErrorString(e_)); cleanup(); return KSC_ECUDA; } } while (0)
    LL_CUDA(cudaMalloc(&Xs, sizeof(float) * ns * d));
    LL_CUDA(cudaMalloc(&cn, sizeof(float) * L));
    LL_CUDA(cudaMalloc(&a, sizeof(int32_t) * ns));
    LL_CUDA(cudaMalloc(&sums, sizeof(double) * L * d));
    LL_CUDA(cudaMalloc(&cnt, sizeof(unsigned long long) * L));
    k_gather_rows<<<grid_for(ns * d), 256, 0, st>>>(X, sample_dev, ns, d, Xs);
    LL_CUDA(cudaMemcpyAsync(C, Xs, sizeof(float) * L * d, cudaMemcpyDeviceToDevice, st));
    for (int it = 0; it < iters; ++it) {
        k_row_sqnorm<<<(L + 255) / 256, 256, 0, st>>>(C, L, d, cn);
        k_assign<<<(unsigned)((ns + AS_T - 1) / AS_T), 256, 0, st>>>(Xs, ns, d, C, cn, L, 0, a, nullptr);
        LL_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * L * d, st));
        LL_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * L, st));
        k_centroid_accum<<<grid_for(ns * d), 256, 0, st>>>(Xs, nullptr, ns, d, a, sums, cnt);
        k_centroid_finish<<<grid_for((int64_t)L * d), 256, 0, st>>>(sums, cnt, C, L, d, C);
        LL_CUDA(cudaGetLastError());
    }
    LL_CUDA(cudaStreamSynchronize(st));
    cleanup();
#undef LL_CUDA
    return rc;
}

}  // namespace ksc

using namespace ksc;

extern "C" {

const char* ksc_last_error(void) { return get_error(); }
const char* ksc_version(void) { return "kscann-gb300 0.1 (sm_103a)"; }

void ksc_index_free(ksc_index* ix) {
    if (!ix) return;
    free_index_memory(ix);
    delete ix;
}

int ksc_index_info(const ksc_index* ix, ksc_index_arrays* a) {
    KSC_CHECK_ARG(ix && a, "null argument");
    a->n = ix->n;
    a->d = ix->d;
    a->nlist = ix->L;
    a->M = ix->M;
    a->metric = ix->metric;
    a->spherical = ix->spherical;
    return KSC_OK;
}

static int finish_common(ksc_index* ix, cudaStream_t st) {
    if (!ix->c_rank_sq) KSC_CUDA(cudaMalloc(&ix->c_rank_sq, sizeof(float) * ix->L));
    k_row_sqnorm<<<(ix->L + 255) / 256, 256, 0, st>>>(ix->c_rank, ix->L, ix->d, ix->c_rank_sq);
    KSC_LAUNCH_CHECK();
    KSC_CUDA(cudaMalloc(&ix->status, sizeof(int32_t) * 4));
    KSC_CUDA(cudaMemsetAsync(ix->status, 0, sizeof(int32_t) * 4, st));
    KSC_CUDA(cudaMalloc(&ix->stats, sizeof(unsigned long long) * 4));
    KSC_CUDA(cudaMemsetAsync(ix->stats, 0, sizeof(unsigned long long) * 4, st));
    KSC_CUDA(cudaStreamSynchronize(st));
    return KSC_OK;
}

static int check_shape(int64_t n, int32_t d, int32_t L, int32_t M, bool shard = false) {
    KSC_CHECK_ARG(n > 0 && n < (1ll << 31), "n must be in [1, 2^31)");
    KSC_CHECK_ARG(d > 0 && d <= KSC_MAX_DIM, "d must be in [1, %d]", KSC_MAX_DIM);
    // a shard holds every list (most of them empty): nlist may exceed its rows
    KSC_CHECK_ARG(L > 0 && L <= KSC_MAX_NLIST && (shard || L <= n), "nlist must be in [1, min(n, %d)]",
                  KSC_MAX_NLIST);
    KSC_CHECK_ARG(M > 0 && M <= KSC_MAX_M && d % M == 0, "M must divide d and be <= %d", KSC_MAX_M);
    return KSC_OK;
}

static int import_arrays(const ksc_index_arrays* a, void* stream, ksc_index** out, bool shard) {
    KSC_CHECK_ARG(a && out && a->X && a->c_rank && a->c_mean && a->codebook && a->codes && a->assign,
                  "null argument");
    KSC_TRY(check_shape(a->n, a->d, a->nlist, a->M, shard));
    KSC_CHECK_ARG(a->metric == KSC_L2 || a->metric == KSC_IP, "bad metric");
    // Every index the device code follows is checked here, on the host,
    // before any device work: codes address 16-entry tables, lists address
    // the list arrays, and the graph preparation and search take a neighbour
    // (or a list's entry) as a position inside its own list, so a neighbour
    // of another list would address codes and visited bits outside the list.
    const int64_t ncodes = a->n * a->M;
    for (int64_t i = 0; i < ncodes; ++i)
        KSC_CHECK_ARG(a->codes[i] < PQ_K, "code %lld is out of range", (long long)i);
    for (int64_t i = 0; i < a->n; ++i)
        KSC_CHECK_ARG(a->assign[i] >= 0 && a->assign[i] < a->nlist, "assignment of row %lld out of range",
                      (long long)i);
    if (a->graph && a->entry) {
        for (int64_t u = 0; u < a->n; ++u)
            for (int e = 0; e < 32; ++e) {
                const int32_t v = a->graph[u * 32 + e];
                KSC_CHECK_ARG(v >= -1 && v < a->n, "neighbour %d of row %lld is out of range", e, (long long)u);
                KSC_CHECK_ARG(v < 0 || a->assign[v] == a->assign[u],
                              "neighbour %d of row %lld is in another list", e, (long long)u);
            }
        for (int32_t p = 0; p < a->nlist; ++p) {
            const int32_t v = a->entry[p];
            KSC_CHECK_ARG(v >= -1 && v < a->n, "graph entry of list %d is out of range", p);
            KSC_CHECK_ARG(v < 0 || a->assign[v] == p, "graph entry of list %d is not in the list", p);
        }
    }
    cudaStream_t st = as_stream(stream);
    ksc_index* ix = new ksc_index();
    ix->n = a->n;
    ix->d = a->d;
    ix->L = a->nlist;
    ix->M = a->M;
    ix->dsub = a->d / a->M;
    ix->metric = a->metric;
    ix->spherical = (a->spherical || a->metric == KSC_IP) ? 1 : 0;
    int rc = KSC_OK;
    uint8_t* codes_dev = nullptr;
    do {
        if ((rc = alloc_copy((void**)&ix->X, a->X, sizeof(float) * ix->n * ix->d, st, cudaMemcpyHostToDevice))) break;
        if ((rc = alloc_copy((void**)&ix->c_rank, a->c_rank, sizeof(float) * ix->L * ix->d, st, cudaMemcpyHostToDevice))) break;
        if ((rc = alloc_copy((void**)&ix->c_mean, a->c_mean, sizeof(float) * ix->L * ix->d, st, cudaMemcpyHostToDevice))) break;
        if ((rc = alloc_copy((void**)&ix->codebook, a->codebook, sizeof(float) * ix->M * PQ_K * ix->dsub, st,
                             cudaMemcpyHostToDevice))) break;
        if ((rc = alloc_copy((void**)&ix->assign, a->assign, sizeof(int32_t) * ix->n, st, cudaMemcpyHostToDevice))) break;
        if ((rc = alloc_copy((void**)&codes_dev, a->codes, (size_t)ix->n * ix->M, st, cudaMemcpyHostToDevice))) break;
        if ((rc = pack_lists(ix, codes_dev, a->assign, st))) break;
        if (a->graph && a->entry) {
            if ((rc = alloc_copy((void**)&ix->graph, a->graph, sizeof(int32_t) * ix->n * 32, st, cudaMemcpyHostToDevice))) break;
            if ((rc = alloc_copy((void**)&ix->entry, a->entry, sizeof(int32_t) * ix->L, st, cudaMemcpyHostToDevice))) break;
            if ((rc = prepare_graph(ix, st))) break;
        }
        rc = finish_common(ix, st);
    } while (0);
    if (codes_dev) cudaFree(codes_dev);
    if (rc != KSC_OK) {
        ksc_index_free(ix);
        return rc;
    }
    *out = ix;
    return KSC_OK;
}

int ksc_index_import(const ksc_index_arrays* a, void* stream, ksc_index** out) {
    return import_arrays(a, stream, out, false);
}

// One shard of a list-partitioned index: the lists p with list_owner[p] ==
// shard keep their members (rows in ascending global id), every other list
// is empty; centroids and codebooks are replicated, so every shard ranks the
// lists and scales the tables (a_q over the whole probe set) as the whole
// index does.  gids maps local rows back to the global ids.
int ksc_index_import_shard(const ksc_index_arrays* full, const int32_t* list_owner, int32_t shard, void* stream,
                           ksc_index** out) {
    KSC_CHECK_ARG(full && list_owner && out && full->X && full->codes && full->assign, "null argument");
    KSC_CHECK_ARG(shard >= 0, "shard must be >= 0");
    KSC_TRY(check_shape(full->n, full->d, full->nlist, full->M));
    for (int32_t p = 0; p < full->nlist; ++p) KSC_CHECK_ARG(list_owner[p] >= 0, "owner of list %d is negative", p);
    std::vector<int32_t> rows;
    for (int64_t i = 0; i < full->n; ++i) {
        const int32_t p = full->assign[i];
        KSC_CHECK_ARG(p >= 0 && p < full->nlist, "assignment of row %lld out of range", (long long)i);
        if (list_owner[p] == shard) rows.push_back((int32_t)i);
    }
    KSC_CHECK_ARG(!rows.empty(), "shard %d holds no vector", shard);
    const int64_t ns = (int64_t)rows.size();
    const int d = full->d, M = full->M;
    std::vector<float> X((size_t)ns * d);
    std::vector<uint8_t> codes((size_t)ns * M);
    std::vector<int32_t> assign(ns);
    for (int64_t r = 0; r < ns; ++r) {
        const int64_t i = rows[r];
        std::copy(full->X + i * d, full->X + (i + 1) * d, X.begin() + r * d);
        std::copy(full->codes + i * M, full->codes + (i + 1) * M, codes.begin() + r * M);
        assign[r] = full->assign[i];
    }
    ksc_index_arrays a = *full;
    a.n = ns;
    a.X = X.data();
    a.codes = codes.data();
    a.assign = assign.data();
    a.graph = nullptr;
    a.entry = nullptr;
    ksc_index* ix = nullptr;
    KSC_TRY(import_arrays(&a, stream, &ix, true));
    if (alloc_copy((void**)&ix->gids, rows.data(), sizeof(int32_t) * ns, as_stream(stream),
                   cudaMemcpyHostToDevice) != KSC_OK ||
        cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) {
        ksc_index_free(ix);
        set_error("shard id map: device copy failed");
        return KSC_ECUDA;
    }
    *out = ix;
    return KSC_OK;
}

int ksc_index_export(const ksc_index* ix, ksc_index_arrays* a) {
    KSC_CHECK_ARG(ix && a, "null argument");
    ksc_index_info(ix, a);
    if (a->X) KSC_CUDA(cudaMemcpy(a->X, ix->X, sizeof(float) * ix->n * ix->d, cudaMemcpyDeviceToHost));
    if (a->c_rank) KSC_CUDA(cudaMemcpy(a->c_rank, ix->c_rank, sizeof(float) * ix->L * ix->d, cudaMemcpyDeviceToHost));
    if (a->c_mean) KSC_CUDA(cudaMemcpy(a->c_mean, ix->c_mean, sizeof(float) * ix->L * ix->d, cudaMemcpyDeviceToHost));
    if (a->codebook)
        KSC_CUDA(cudaMemcpy(a->codebook, ix->codebook, sizeof(float) * ix->M * PQ_K * ix->dsub, cudaMemcpyDeviceToHost));
    if (a->assign) KSC_CUDA(cudaMemcpy(a->assign, ix->assign, sizeof(int32_t) * ix->n, cudaMemcpyDeviceToHost));
    if (a->codes) {
        uint8_t* codes_dev = nullptr;
        KSC_CUDA(cudaMalloc(&codes_dev, (size_t)ix->n * ix->M));
        k_unpack<<<grid_for(ix->nblocks * 32 * ix->M), 256>>>(ix->blk_ids, ix->nblocks, ix->M, ix->blk_codes,
                                                              codes_dev);
        cudaError_t e = cudaMemcpy(a->codes, codes_dev, (size_t)ix->n * ix->M, cudaMemcpyDeviceToHost);
        cudaFree(codes_dev);
        KSC_CUDA(e);
    }
    if (a->graph && ix->graph) KSC_CUDA(cudaMemcpy(a->graph, ix->graph, sizeof(int32_t) * ix->n * 32, cudaMemcpyDeviceToHost));
    if (a->entry && ix->entry) KSC_CUDA(cudaMemcpy(a->entry, ix->entry, sizeof(int32_t) * ix->L, cudaMemcpyDeviceToHost));
    return KSC_OK;
}

// Component filtration (Sec. 4.3; Alg. 1 FilterComponents): the index is
// built on the kept dimensions -- the sub-vector width d / M is kept, so the
// filtered index has ceil(kept / (d / M)) subspaces, the last completed with
// zero dimensions -- and holds the full vectors for the re-rank.
static int build_filtered(const float* X_dev, int64_t n, int32_t d, int32_t nlist, int32_t M, int32_t nbits,
                          ksc_metric metric, const ksc_build_opts* opts, void* stream, ksc_index** out) {
    KSC_TRY(check_shape(n, d, nlist, M));
    cudaStream_t st = as_stream(stream);
    const double thr = opts->filter_threshold;
    std::vector<double> frac(d);
    double* stats = nullptr;
    KSC_CUDA(cudaMalloc(&stats, sizeof(double) * 3 * d));
    int rc = component_stats(X_dev, n, d, stats, stats + d, stats + 2 * d, st);
    if (rc == KSC_OK && cudaMemcpy(frac.data(), stats + 2 * d, sizeof(double) * d, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("reading the component statistics failed");
        rc = KSC_ECUDA;
    }
    cudaFree(stats);
    KSC_TRY(rc);
    std::vector<int32_t> dims;
    for (int t = 0; t < d; ++t)
        if (frac[t] <= thr) dims.push_back(t);
    KSC_CHECK_ARG(!dims.empty(), "component filtration kept no dimension (threshold %g)", thr);
    const int dsub = d / M;
    const int Mf = (int)((dims.size() + dsub - 1) / dsub);
    while ((int)dims.size() < Mf * dsub) dims.push_back(-1);
    const int dw = Mf * dsub;
    float* Xw = nullptr;
    int32_t* dims_dev = nullptr;
    KSC_CUDA(cudaMalloc(&dims_dev, sizeof(int32_t) * dw));
    cudaError_t e = cudaMemcpy(dims_dev, dims.data(), sizeof(int32_t) * dw, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&Xw, sizeof(float) * n * dw);
    if (e != cudaSuccess) {
        cudaFree(dims_dev);
        set_error("component filtration: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? KSC_ENOMEM : KSC_ECUDA;
    }
    rc = gather_dims(X_dev, n, d, dims_dev, dw, Xw, st);
    ksc_build_opts inner = *opts;
    inner.filter_threshold = 0.f;
    ksc_index* ix = nullptr;
    if (rc == KSC_OK) rc = ksc_build_index(Xw, n, dw, nlist, Mf, nbits, metric, &inner, stream, &ix);
    cudaStreamSynchronize(st);
    cudaFree(Xw);
    if (rc == KSC_OK) {
        ix->dims = dims_dev;
        dims_dev = nullptr;
        ix->h_dims = dims;
        ix->d_rr = d;
        e = cudaMalloc(&ix->X_rr, sizeof(float) * n * d);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ix->X_rr, X_dev, sizeof(float) * n * d, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            set_error("component filtration: %s", cudaGetErrorString(e));
            rc = e == cudaErrorMemoryAllocation ? KSC_ENOMEM : KSC_ECUDA;
            ksc_index_free(ix);
            ix = nullptr;
        }
    }
    if (dims_dev) cudaFree(dims_dev);
    if (rc == KSC_OK) *out = ix;
    return rc;
}

int ksc_build_index(const float* X_dev, int64_t n, int32_t d, int32_t nlist, int32_t M, int32_t nbits,
                    ksc_metric metric, const ksc_build_opts* opts, void* stream, ksc_index** out) {
    KSC_CHECK_ARG(X_dev && out, "null argument");
    if (opts && opts->filter_threshold > 0.f) return build_filtered(X_dev, n, d, nlist, M, nbits, metric, opts, stream, out);
    if (nbits != 4) {
        set_error("only 4-bit PQ codes (K = 16) are supported, got nbits = %d", nbits);
        return KSC_EUNSUPPORTED;
    }
    KSC_TRY(check_shape(n, d, nlist, M));
    KSC_CHECK_ARG(metric == KSC_L2 || metric == KSC_IP, "bad metric");
    cudaStream_t st = as_stream(stream);
    const int iters = (opts && opts->kmeans_iters > 0) ? opts->kmeans_iters : 20;
    const int spherical = (metric == KSC_IP || (opts && opts->spherical)) ? 1 : 0;
    std::vector<int64_t> perm;
    if (opts && opts->perm_host) {
        perm.assign(opts->perm_host, opts->perm_host + n);
    } else {
        host_perm(n, opts ? opts->seed : 0x5eed, perm);
    }
    ksc_index* ix = new ksc_index();
    ix->n = n; ix->d = d; ix->L = nlist; ix->M = M; ix->dsub = d / M;
    ix->metric = metric; ix->spherical = spherical;
    const int64_t ns = n < 256ll * nlist ? n : 256ll * nlist;
    const int64_t npq = n < 65536 ? n : 65536;
    int64_t* perm_dev = nullptr;
    uint8_t* codes_dev = nullptr;
    float* Rs = nullptr;
    double* sums = nullptr;
    unsigned long long* cnt = nullptr;
    uint8_t* pcodes = nullptr;
    int rc = KSC_OK;
    std::vector<int32_t> assign_host(n);
    do {
#define B_CUDA(call) { cudaError_t e_ = (call); if (e_ != cudaSuccess) { set_error("%s: %s", #call, cudaGetErrorString(e_)); rc = e_ == cudaErrorMemoryAllocation ? KSC_ENOMEM : KSC_ECUDA; break; } }
        B_CUDA(cudaMalloc(&ix->X, sizeof(float) * n * d));
        B_CUDA(cudaMemcpyAsync(ix->X, X_dev, sizeof(float) * n * d, cudaMemcpyDeviceToDevice, st));
        B_CUDA(cudaMalloc(&perm_dev, sizeof(int64_t) * n));
        B_CUDA(cudaMemcpyAsync(perm_dev, perm.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
        B_CUDA(cudaMalloc(&ix->c_rank, sizeof(float) * nlist * d));
        B_CUDA(cudaMalloc(&ix->c_mean, sizeof(float) * nlist * d));
        B_CUDA(cudaMalloc(&ix->c_rank_sq, sizeof(float) * nlist));
        // 1. coarse quantiser
        if ((rc = lloyd(ix->X, perm_dev, ns, d, nlist, iters, ix->c_mean, st))) break;
        B_CUDA(cudaMemcpyAsync(ix->c_rank, ix->c_mean, sizeof(float) * nlist * d, cudaMemcpyDeviceToDevice, st));
        if (spherical) k_normalise_rows<<<(nlist + 255) / 256, 256, 0, st>>>(ix->c_rank, nlist, d);
        k_row_sqnorm<<<(nlist + 255) / 256, 256, 0, st>>>(ix->c_rank, nlist, d, ix->c_rank_sq);
        // 2. list of every vector by the ranking score
        B_CUDA(cudaMalloc(&ix->assign, sizeof(int32_t) * n));
        k_assign<<<(unsigned)((n + AS_T - 1) / AS_T), 256, 0, st>>>(ix->X, n, d, ix->c_rank, ix->c_rank_sq, nlist,
                                                                    spherical, ix->assign, nullptr);
        // 3. mean centroids of the lists (Sec. 4.6.1)
        B_CUDA(cudaMalloc(&sums, sizeof(double) * (size_t)nlist * d));
        B_CUDA(cudaMalloc(&cnt, sizeof(unsigned long long) * nlist));
        B_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * (size_t)nlist * d, st));
        B_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * nlist, st));
        k_centroid_accum<<<grid_for(n * d), 256, 0, st>>>(ix->X, nullptr, n, d, ix->assign, sums, cnt);
        // (empty list: keeps its Lloyd centroid, already in c_mean)
        k_centroid_finish<<<grid_for((int64_t)nlist * d), 256, 0, st>>>(sums, cnt, ix->c_mean, nlist, d, ix->c_mean);
        B_CUDA(cudaGetLastError());
        // 4. PQ codebooks on the residuals of the first npq permuted rows
        B_CUDA(cudaMalloc(&Rs, sizeof(float) * npq * d));
        k_residual<<<grid_for(npq * d), 256, 0, st>>>(ix->X, perm_dev, npq, d, ix->assign, ix->c_mean, Rs);
        B_CUDA(cudaMalloc(&ix->codebook, sizeof(float) * M * PQ_K * ix->dsub));
        B_CUDA(cudaMalloc(&pcodes, (size_t)npq * M));
        cudaFree(sums); sums = nullptr;
        cudaFree(cnt); cnt = nullptr;
        B_CUDA(cudaMalloc(&sums, sizeof(double) * M * PQ_K * ix->dsub));
        B_CUDA(cudaMalloc(&cnt, sizeof(unsigned long long) * M * PQ_K));
        k_pq_init<<<grid_for((int64_t)M * PQ_K * ix->dsub), 256, 0, st>>>(Rs, d, M, ix->dsub, ix->codebook);
        for (int it = 0; it < iters; ++it) {
            k_pq_encode<<<grid_for(npq * M), 256, 0, st>>>(Rs, nullptr, nullptr, nullptr, npq, d, M, ix->dsub,
                                                           ix->codebook, pcodes);
            B_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * M * PQ_K * ix->dsub, st));
            B_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * M * PQ_K, st));
            k_pq_accum<<<grid_for(npq * d), 256, 0, st>>>(Rs, npq, d, M, ix->dsub, pcodes, sums, cnt);
            k_pq_finish<<<grid_for((int64_t)M * PQ_K * ix->dsub), 256, 0, st>>>(sums, cnt, M, ix->dsub, ix->codebook);
        }
        B_CUDA(cudaGetLastError());
        if (rc) break;
        // 5. encode every vector and pack the lists into blocks
        B_CUDA(cudaMalloc(&codes_dev, (size_t)n * M));
        k_pq_encode<<<grid_for(n * M), 256, 0, st>>>(nullptr, ix->X, ix->assign, ix->c_mean, n, d, M, ix->dsub,
                                                     ix->codebook, codes_dev);
        B_CUDA(cudaGetLastError());
        B_CUDA(cudaMemcpyAsync(assign_host.data(), ix->assign, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
        B_CUDA(cudaStreamSynchronize(st));
        if ((rc = pack_lists(ix, codes_dev, assign_host.data(), st))) break;
        if ((rc = finish_common(ix, st))) break;
        if (opts && opts->build_graph) {
            if ((rc = ksc::build_graph(ix, st))) break;
        }
#undef B_CUDA
    } while (0);
    cudaFree(perm_dev); cudaFree(codes_dev); cudaFree(Rs); cudaFree(sums); cudaFree(cnt); cudaFree(pcodes);
    if (rc != KSC_OK) {
        ksc_index_free(ix);
        return rc;
    }
    *out = ix;
    return KSC_OK;
}

}  // extern "C"

extern "C" int ksc_index_dims(ksc_index* ix, int32_t* dims_host, int32_t* d_full_host) {
    KSC_CHECK_ARG(ix && d_full_host, "null argument");
    *d_full_host = ix->X_rr ? ix->d_rr : ix->d;
    if (dims_host)
        for (int j = 0; j < ix->d; ++j) dims_host[j] = ix->X_rr ? ix->h_dims[j] : j;
    return KSC_OK;
}

extern "C" int ksc_component_stats(const float* X_dev, int64_t n, int32_t d, double* mu_dev, double* sd_dev,
                                   double* frac_dev, void* stream) {
    KSC_CHECK_ARG(X_dev && mu_dev && sd_dev && frac_dev && n > 0 && d > 0, "bad argument");
    return ksc::component_stats(X_dev, n, d, mu_dev, sd_dev, frac_dev, ksc::as_stream(stream));
}

// A second handle on the same index data with its own search workspace,
// status word, counters and stage events, so that searches on different
// streams can run at the same time (one handle each).
extern "C" int ksc_index_view(ksc_index* ix, ksc_index** out) {
    KSC_CHECK_ARG(ix && out, "null argument");
    ksc_index* v = new ksc_index(*ix);  // the shared arrays, models and host mirrors
    v->parent = ix;
    ksc::Buffer* bufs[64];
    const int nb = workspace_buffers(v, bufs);
    for (int i = 0; i < nb; ++i) *bufs[i] = ksc::Buffer{};
    for (int i = 0; i <= KSC_NUM_STAGES; ++i) {
        v->ev[i] = nullptr;
        v->ev_used[i] = false;
    }
    v->prof = false;
    v->launches = 0;
    v->status = nullptr;
    v->stats = nullptr;
    cudaError_t e = cudaMalloc(&v->status, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&v->stats, sizeof(unsigned long long) * 4);
    if (e == cudaSuccess) e = cudaMemset(v->status, 0, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(v->stats, 0, sizeof(unsigned long long) * 4);
    if (e != cudaSuccess) {
        ksc::set_error("ksc_index_view: %s", cudaGetErrorString(e));
        ksc_index_free(v);
        return e == cudaErrorMemoryAllocation ? KSC_ENOMEM : KSC_ECUDA;
    }
    *out = v;
    return KSC_OK;
}
