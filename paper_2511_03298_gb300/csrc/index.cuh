// Device-resident IVF-PQ index (Alg. 1 output) and its search workspace.
#pragma once

#include <vector>

#include "common.cuh"

// Block layout of the 4-bit codes (GPU-internal): every list is cut into
// blocks of 32 vectors (the paper's SIMD data blocks, Sec. 4.5.3).  A block
// stores M chunks of 16 bytes, one per subspace j (subspace-major); byte i
// of chunk j holds code_j of vector 2i in its low nibble and of vector 2i+1
// in its high nibble.  Hence the 32-bit word w of chunk j carries the codes
// of vectors 8w..8w+7, vector 8w+t in bits 4t..4t+3.
constexpr int BLOCK_VECS = 32;
constexpr int PQ_K = 16;

struct ksc_index {
    int64_t n = 0;
    int32_t d = 0, L = 0, M = 0, dsub = 0, metric = KSC_L2, spherical = 0;
    int64_t nblocks = 0;
    int32_t max_list = 0;
    // device arrays
    float* X = nullptr;          // [n x d]
    float* c_rank = nullptr;     // [L x d]
    float* c_rank_sq = nullptr;  // [L] ||c_rank||^2
    float* c_mean = nullptr;     // [L x d]
    float* codebook = nullptr;   // [M x 16 x dsub]
    int64_t* list_boff = nullptr;  // [L + 1] first block of each list
    int32_t* list_n = nullptr;     // [L] list sizes
    int32_t* blk_ids = nullptr;    // [nblocks x 32] ids, -1 padding
    uint8_t* blk_codes = nullptr;  // [nblocks x M x 16]
    int32_t* assign = nullptr;     // [n]
    int32_t* blk_list = nullptr;   // [nblocks] list of each block
    int32_t* graph = nullptr;      // [n x 32] optional: neighbours by id (interchange form)
    int32_t* entry = nullptr;      // [L] optional: graph entry by id
    int32_t* nbr_pos = nullptr;    // [nblocks x 32 x 32] neighbours as list positions
    uint8_t* nbr_codes = nullptr;  // [nblocks x 32 x M x 16] neighbour codes, one block per node
    int32_t* entry_pos = nullptr;  // [L] graph entry as a list position
    void* X_bf16 = nullptr;        // [n x d] BF16 rows (precision variant, made on first use)
    void* X_fp8 = nullptr;         // [n x d] FP8 e4m3 rows
    float* X_scale = nullptr;      // [n] their per-row scales
    void* X_u8 = nullptr;          // [n x d] U8 rows when every coordinate is an integer in [0, 255] (exact)
    int x_u8_state = 0;            // 0 not checked, 1 X_u8 holds the rows exactly, -1 they do not fit bytes
    float2* X_band = nullptr;      // [n] per re-rank row: bounds of its norm and of its BF16 rounding error's norm (made on first use)
    int32_t* status = nullptr;     // device status word
    unsigned long long* stats = nullptr;  // [4] counters of the last search
    // host mirrors
    std::vector<int64_t> h_boff;   // [L + 1]
    std::vector<int32_t> h_n;      // [L]
    // tensor-core ranking: BF16 copy of c_rank [L x Kp], its TMA map, max ||c||
    void* c_rank_bf16 = nullptr;
    alignas(64) unsigned char map_c[128] = {};
    float c_rank_max_norm = 0.f;
    bool tc_fp16 = false;  // 16-bit operand type of the tensor-core ranking
    // FP8 ranking option: e4m3 copy of c_rank [L x Kp8] with power-of-two row
    // scales [L] and its TMA map (made on first use)
    void* c_rank_f8 = nullptr;
    float* c_rank_f8_scale = nullptr;
    alignas(64) unsigned char map_c8[128] = {};
    // learned nprobe / rerank predictor (Sec. 4.2.1-4.2.2)
    float* mlp_w = nullptr;  // [KSC_MLP_NPARAMS] FP32
    ksc_adaptive_params mlp_prm = {};
    // predictive cluster pruning (Sec. 4.2.3): per-list statistics, vectors, model
    float* pr_stats = nullptr;  // [L x KSC_PRUNE_STATS]
    float* pr_vecs = nullptr;   // [L x 3 x d] v1, v2, mean outlier offset
    float* pr_model = nullptr;  // [KSC_PRUNE_MODEL] weights, feature means, feature stds
    bool pr_have_stats = false;
    float pr_theta = -1.f;      // applied by the adaptive search when >= 0
    // component filtration (Sec. 4.3): the index lives on the kept dimensions
    // (d, X); queries arrive with d_rr dimensions and the re-rank reads X_rr
    int32_t* dims = nullptr;     // [d] query dimension of each working one (-1: zero)
    std::vector<int32_t> h_dims;
    float* X_rr = nullptr;       // [n x d_rr] full vectors (null: no filtration)
    int32_t d_rr = 0;
    // list sharding (ksc_index_import_shard): global id of each local row,
    // ascending, so (distance, local id) orders keys as (distance, global id)
    int32_t* gids = nullptr;  // [n]
    // a view (ksc_index_view): the handle it came from, whose arrays it shares
    const ksc_index* parent = nullptr;
    // stage timing (ksc_profile_enable)
    bool prof = false;
    cudaEvent_t ev[KSC_NUM_STAGES + 1] = {};
    bool ev_used[KSC_NUM_STAGES + 1] = {};
    int32_t launches = 0;
    // search workspace
    ksc::Buffer ws_scores, ws_probes, ws_lut, ws_bias, ws_scale, ws_range, ws_thr, ws_cnt,
        ws_cand, ws_topr, ws_nprobe, ws_rerank, ws_items, ws_misc, ws_qbf16, ws_err, ws_feat, ws_rscore, ws_full, ws_topr2, ws_flag,
        ws_redo, ws_pprobes, ws_pn, ws_pprob, ws_qf;
};

// The vectors the exact re-rank reads and their width: the full vectors when
// component filtration dropped dimensions (Alg. 2 re-ranks with the
// unfiltered query), else X.
inline const float* rr_X(const ksc_index* ix) { return ix->X_rr ? ix->X_rr : ix->X; }
inline int rr_d(const ksc_index* ix) { return ix->X_rr ? ix->d_rr : ix->d; }

namespace ksc {
// Fill blk_ids / blk_codes / list tables from unpacked codes [n x M] (device)
// and the list of each vector (host copy), members in ascending id order.
int pack_lists(ksc_index* ix, const uint8_t* codes_dev, const int32_t* assign_host, cudaStream_t st);
int free_index_memory(ksc_index* ix);
// Tensor-core list scores (rank_tc.cu): approximate scores [nq x L] and a
// per-query bound err [nq] on their error.
bool tc_rank_supported(const ksc_index* ix);
int rank_scores_tc(ksc_index* ix, const float* Q, int64_t nq, float* scores, float* err, cudaStream_t st);
// The same from e4m3 operands with per-row power-of-two scales (FP8 option).
int rank_scores_tc8(ksc_index* ix, const float* Q, int64_t nq, float* scores, float* err, cudaStream_t st);
// Per-query error bound of the list scores (tensor-core or FP32 path).
int score_err(ksc_index* ix, const float* Q, int64_t nq, bool tensor_cores, float* err, cudaStream_t st);
// Gather of rows src[idx[r]] (width d floats) into dst (index.cu).
__global__ void k_gather_rows(const float* __restrict__ X, const int64_t* __restrict__ idx, int64_t cnt, int d,
                              float* __restrict__ out);
// MLP kernels (mlp.cu).
int mlp_grad(const float* w, const float* x, const float* y, int64_t B, float* grad, float* loss, cudaStream_t st);
int mlp_infer(const float* w, const float* x, int64_t B, const ksc_adaptive_params& prm, float* prob,
              int32_t* nprobe, int32_t* rerank, cudaStream_t st);
int mlp_features(const float* scores, int64_t nq, int ld, int spherical, float* feats, cudaStream_t st);
// Features and inference in one kernel (the adaptive search): settings per query.
int mlp_infer_scores(const float* w, const float* scores, int ld, int spherical, int64_t B,
                     const ksc_adaptive_params& prm, int32_t* nprobe, int32_t* rerank, cudaStream_t st);
int mlp_hits(const float* dists, int64_t nq, int k, const float* kth, int ip, int32_t* hits, cudaStream_t st);
int mlp_adam(float* w, const float* g, float* m, float* v, int t, float lr, cudaStream_t st);
int mlp_adam_n(float* w, const float* g, float* m, float* v, int n, int t, float lr, cudaStream_t st);
int prune_mlp_grad(const float* w, const float* x, const float* y, int64_t B, float* grad, float* loss,
                   cudaStream_t st);
// Predictive cluster pruning (prune.cu): per-list statistics; features /
// keep probabilities / pruned probe lists of (query, rank) rows; labels;
// feature standardisation (moments into the model) and training targets.
int prune_stats(ksc_index* ix, int iters, cudaStream_t st);
int prune_rows(ksc_index* ix, const float* Q, int64_t nq, const int32_t* probes, int Pmax, const int32_t* nprobe,
               int P, float theta, float* feats, float* prob, int32_t* probes_out, int32_t* nprobe_out,
               cudaStream_t st);
int prune_labels(ksc_index* ix, const int64_t* ids, const float* dists, int64_t nq, int k, const float* kth,
                 const int32_t* probes, int Pmax, int P, float* label, cudaStream_t st);
int prune_standardise(float* x, int64_t rows, float* model, cudaStream_t st);
int prune_targets(const float* lab, int64_t rows, float* y, cudaStream_t st);
// Component filtration (filter.cu): column statistics, dimension gather.
int component_stats(const float* X, int64_t n, int d, double* mu, double* sd, double* frac, cudaStream_t st);
int gather_dims(const float* A, int64_t rows, int d, const int32_t* dims, int dw, float* out, cudaStream_t st);
// List sharding (search.cu): steps a1 .. a5 of a fixed-nprobe search into
// sorted keys [nq x R] (local ids), and the exact re-rank of given keys.
int search_keys(ksc_index* ix, const float* Q, int64_t nq, int nprobe, int rerank, const ksc_search_opts* opts,
                uint64_t* keys, cudaStream_t st);
int rerank_keys(ksc_index* ix, const float* Q, int64_t nq, int k, const uint64_t* keys, int R, int64_t* ids,
                float* dists, cudaStream_t st);
// Per-list 32-NN graphs and entry points for the hybrid search (Sec. 4.4).
int build_graph(ksc_index* ix, cudaStream_t st);
// Search form (nbr_pos, nbr_codes, entry_pos) of graph / entry (hybrid.cu).
int prepare_graph(ksc_index* ix, cudaStream_t st);
}  // namespace ksc
