// Index persistence: ksc_index_save / ksc_index_load.
//
// One binary file, little-endian, a 64-byte header then the arrays in a fixed
// order.  Always present: the interchange arrays of ksc_index_export (vectors,
// both centroid sets, codebook, unpacked codes, list of each vector).  Present
// when the index holds them (a header flag each): the intra-list graph and its
// entries, the learned predictor's weights and parameters, the pruning
// statistics and model (and its threshold), and the component-filtration state
// (kept dimensions and full vectors).  Loading validates the whole file on the
// host -- header, exact size, every code, list, neighbour and dimension index --
// before any device work, then builds the index through the same path as
// ksc_index_import and attaches the optional state.
#include <cstdio>
#include <cstring>
#include <vector>

#include "index.cuh"

namespace ksc {
namespace {

constexpr char MAGIC[8] = {'K', 'S', 'C', 'I', 'D', 'X', '0', '1'};
enum : int32_t { F_GRAPH = 1, F_PREDICTOR = 2, F_PRUNE_STATS = 4, F_PRUNE_MODEL = 8, F_FILTER = 16 };
constexpr int32_t F_ALL = F_GRAPH | F_PREDICTOR | F_PRUNE_STATS | F_PRUNE_MODEL | F_FILTER;

struct FileHeader {
    char magic[8];
    int64_t n;
    int32_t d, nlist, M, metric, spherical, flags;
    int32_t d_full;       // filtration: dimensions of the full vectors (else 0)
    int32_t prm_bytes;    // sizeof(ksc_adaptive_params) of the writer
    int32_t reserved[4];  // zero
};
static_assert(sizeof(FileHeader) == 64, "file header layout");

// Byte sizes of the sections a header announces, in file order.
struct Sections {
    size_t X, c_rank, c_mean, codebook, codes, assign, graph, entry, mlp_w, mlp_prm, pr_stats, pr_vecs, pr_model,
        pr_theta, dims, X_full;
    size_t total() const {
        return sizeof(FileHeader) + X + c_rank + c_mean + codebook + codes + assign + graph + entry + mlp_w + mlp_prm +
               pr_stats + pr_vecs + pr_model + pr_theta + dims + X_full;
    }
};

Sections sections_of(const FileHeader& h) {
    const size_t n = (size_t)h.n, d = (size_t)h.d, L = (size_t)h.nlist, M = (size_t)h.M;
    Sections s{};
    s.X = sizeof(float) * n * d;
    s.c_rank = s.c_mean = sizeof(float) * L * d;
    s.codebook = sizeof(float) * M * PQ_K * (d / M);
    s.codes = n * M;
    s.assign = sizeof(int32_t) * n;
    if (h.flags & F_GRAPH) {
        s.graph = sizeof(int32_t) * n * 32;
        s.entry = sizeof(int32_t) * L;
    }
    if (h.flags & F_PREDICTOR) {
        s.mlp_w = sizeof(float) * KSC_MLP_NPARAMS;
        s.mlp_prm = sizeof(ksc_adaptive_params);
    }
    if (h.flags & F_PRUNE_STATS) {
        s.pr_stats = sizeof(float) * L * KSC_PRUNE_STATS;
        s.pr_vecs = sizeof(float) * L * 3 * d;
    }
    if (h.flags & F_PRUNE_MODEL) {
        s.pr_model = sizeof(float) * KSC_PRUNE_MODEL;
        s.pr_theta = sizeof(float);
    }
    if (h.flags & F_FILTER) {
        s.dims = sizeof(int32_t) * d;
        s.X_full = sizeof(float) * n * (size_t)h.d_full;
    }
    return s;
}

struct File {
    FILE* f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

bool put(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool get(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

template <class T>
int d2h(std::vector<T>& v, const void* dev, size_t count) {
    v.resize(count);
    KSC_CUDA(cudaMemcpy(v.data(), dev, sizeof(T) * count, cudaMemcpyDeviceToHost));
    return KSC_OK;
}

}  // namespace
}  // namespace ksc

using namespace ksc;

extern "C" {

int ksc_index_save(const ksc_index* ix_in, const char* path) {
    KSC_CHECK_ARG(ix_in && path, "null argument");
    // a view holds the arrays and models of the index it came from
    ksc_index* ix = const_cast<ksc_index*>(ix_in->parent ? ix_in->parent : ix_in);
    KSC_CUDA(cudaDeviceSynchronize());
    FileHeader h{};
    std::memcpy(h.magic, MAGIC, sizeof(MAGIC));
    h.n = ix->n;
    h.d = ix->d;
    h.nlist = ix->L;
    h.M = ix->M;
    h.metric = ix->metric;
    h.spherical = ix->spherical;
    h.flags = (ix->graph && ix->entry ? F_GRAPH : 0) | (ix->mlp_w ? F_PREDICTOR : 0) |
              (ix->pr_have_stats ? F_PRUNE_STATS : 0) | (ix->pr_model ? F_PRUNE_MODEL : 0) |
              (ix->X_rr ? F_FILTER : 0);
    h.d_full = ix->X_rr ? ix->d_rr : 0;
    h.prm_bytes = (int32_t)sizeof(ksc_adaptive_params);
    const Sections s = sections_of(h);
    // the interchange arrays
    std::vector<float> X(s.X / 4), c_rank(s.c_rank / 4), c_mean(s.c_mean / 4), codebook(s.codebook / 4);
    std::vector<uint8_t> codes(s.codes);
    std::vector<int32_t> assign(s.assign / 4), graph(s.graph / 4), entry(s.entry / 4);
    ksc_index_arrays a{};
    a.X = X.data();
    a.c_rank = c_rank.data();
    a.c_mean = c_mean.data();
    a.codebook = codebook.data();
    a.codes = codes.data();
    a.assign = assign.data();
    a.graph = (h.flags & F_GRAPH) ? graph.data() : nullptr;
    a.entry = (h.flags & F_GRAPH) ? entry.data() : nullptr;
    KSC_TRY(ksc_index_export(ix, &a));
    std::vector<float> mlp_w, pr_stats, pr_vecs, pr_model, X_full;
    if (h.flags & F_PREDICTOR) KSC_TRY(d2h(mlp_w, ix->mlp_w, KSC_MLP_NPARAMS));
    if (h.flags & F_PRUNE_STATS) {
        KSC_TRY(d2h(pr_stats, ix->pr_stats, (size_t)ix->L * KSC_PRUNE_STATS));
        KSC_TRY(d2h(pr_vecs, ix->pr_vecs, (size_t)ix->L * 3 * ix->d));
    }
    if (h.flags & F_PRUNE_MODEL) KSC_TRY(d2h(pr_model, ix->pr_model, KSC_PRUNE_MODEL));
    if (h.flags & F_FILTER) {
        KSC_CHECK_STATE((int)ix->h_dims.size() == ix->d, "inconsistent component-filtration state");
        KSC_TRY(d2h(X_full, ix->X_rr, (size_t)ix->n * ix->d_rr));
    }
    File file;
    file.f = std::fopen(path, "wb");
    KSC_CHECK_ARG(file.f, "cannot open %s for writing", path);
    const float theta = ix->pr_theta;
    bool ok = put(file.f, &h, sizeof(h)) && put(file.f, X.data(), s.X) && put(file.f, c_rank.data(), s.c_rank) &&
              put(file.f, c_mean.data(), s.c_mean) && put(file.f, codebook.data(), s.codebook) &&
              put(file.f, codes.data(), s.codes) && put(file.f, assign.data(), s.assign) &&
              put(file.f, graph.data(), s.graph) && put(file.f, entry.data(), s.entry) &&
              put(file.f, mlp_w.data(), s.mlp_w) && put(file.f, &ix->mlp_prm, s.mlp_prm) &&
              put(file.f, pr_stats.data(), s.pr_stats) && put(file.f, pr_vecs.data(), s.pr_vecs) &&
              put(file.f, pr_model.data(), s.pr_model) && put(file.f, &theta, s.pr_theta) &&
              put(file.f, ix->h_dims.data(), s.dims) && put(file.f, X_full.data(), s.X_full);
    ok = (std::fclose(file.f) == 0) && ok;
    file.f = nullptr;
    if (!ok) {
        std::remove(path);
        set_error("writing %s failed", path);
        return KSC_EINVAL;
    }
    return KSC_OK;
}

int ksc_index_load(const char* path, void* stream, ksc_index** out) {
    KSC_CHECK_ARG(path && out, "null argument");
    File file;
    file.f = std::fopen(path, "rb");
    KSC_CHECK_ARG(file.f, "cannot open %s", path);
    FileHeader h{};
    KSC_CHECK_ARG(get(file.f, &h, sizeof(h)) && std::memcmp(h.magic, MAGIC, sizeof(MAGIC)) == 0,
                  "%s is not an index file of this library", path);
    KSC_CHECK_ARG(h.n > 0 && h.n < (1ll << 31) && h.d > 0 && h.d <= KSC_MAX_DIM && h.nlist > 0 &&
                      h.nlist <= KSC_MAX_NLIST && h.nlist <= h.n && h.M > 0 && h.M <= KSC_MAX_M && h.d % h.M == 0,
                  "%s: bad index shape", path);
    KSC_CHECK_ARG(h.metric == KSC_L2 || h.metric == KSC_IP, "%s: bad metric", path);
    KSC_CHECK_ARG((h.flags & ~F_ALL) == 0, "%s: unknown sections", path);
    KSC_CHECK_ARG(h.prm_bytes == (int32_t)sizeof(ksc_adaptive_params), "%s: written by another version", path);
    KSC_CHECK_ARG((h.flags & F_FILTER) ? (h.d_full > 0 && h.d_full <= KSC_MAX_DIM) : h.d_full == 0,
                  "%s: bad filtration dimensions", path);
    const Sections s = sections_of(h);
    KSC_CHECK_ARG(std::fseek(file.f, 0, SEEK_END) == 0, "%s: cannot seek", path);
    const long long size = std::ftell(file.f);
    KSC_CHECK_ARG(size >= 0 && (size_t)size == s.total(), "%s: %lld bytes, the header announces %zu", path, size,
                  s.total());
    KSC_CHECK_ARG(std::fseek(file.f, (long)sizeof(FileHeader), SEEK_SET) == 0, "%s: cannot seek", path);
    std::vector<float> X(s.X / 4), c_rank(s.c_rank / 4), c_mean(s.c_mean / 4), codebook(s.codebook / 4);
    std::vector<uint8_t> codes(s.codes);
    std::vector<int32_t> assign(s.assign / 4), graph(s.graph / 4), entry(s.entry / 4), dims(s.dims / 4);
    std::vector<float> mlp_w(s.mlp_w / 4), pr_stats(s.pr_stats / 4), pr_vecs(s.pr_vecs / 4), pr_model(s.pr_model / 4),
        X_full(s.X_full / 4);
    ksc_adaptive_params prm{};
    float theta = -1.f;
    const bool ok = get(file.f, X.data(), s.X) && get(file.f, c_rank.data(), s.c_rank) &&
                    get(file.f, c_mean.data(), s.c_mean) && get(file.f, codebook.data(), s.codebook) &&
                    get(file.f, codes.data(), s.codes) && get(file.f, assign.data(), s.assign) &&
                    get(file.f, graph.data(), s.graph) && get(file.f, entry.data(), s.entry) &&
                    get(file.f, mlp_w.data(), s.mlp_w) && get(file.f, &prm, s.mlp_prm) &&
                    get(file.f, pr_stats.data(), s.pr_stats) && get(file.f, pr_vecs.data(), s.pr_vecs) &&
                    get(file.f, pr_model.data(), s.pr_model) && get(file.f, &theta, s.pr_theta) &&
                    get(file.f, dims.data(), s.dims) && get(file.f, X_full.data(), s.X_full);
    KSC_CHECK_ARG(ok, "%s: read failed", path);
    // index ranges; list membership of neighbours and entries is checked by
    // ksc_index_import below, still before any device work
    for (uint8_t c : codes) KSC_CHECK_ARG(c < PQ_K, "%s: a code is out of range", path);
    for (int32_t p : assign) KSC_CHECK_ARG(p >= 0 && p < h.nlist, "%s: a list index is out of range", path);
    for (int32_t v : graph) KSC_CHECK_ARG(v >= -1 && v < h.n, "%s: a neighbour index is out of range", path);
    for (int32_t v : entry) KSC_CHECK_ARG(v >= -1 && v < h.n, "%s: a graph entry is out of range", path);
    for (int32_t t : dims) KSC_CHECK_ARG(t >= -1 && t < h.d_full, "%s: a kept dimension is out of range", path);
    ksc_index_arrays a{};
    a.n = h.n;
    a.d = h.d;
    a.nlist = h.nlist;
    a.M = h.M;
    a.metric = h.metric;
    a.spherical = h.spherical;
    a.X = X.data();
    a.c_rank = c_rank.data();
    a.c_mean = c_mean.data();
    a.codebook = codebook.data();
    a.codes = codes.data();
    a.assign = assign.data();
    a.graph = (h.flags & F_GRAPH) ? graph.data() : nullptr;
    a.entry = (h.flags & F_GRAPH) ? entry.data() : nullptr;
    ksc_index* ix = nullptr;
    KSC_TRY(ksc_index_import(&a, stream, &ix));
    int rc = KSC_OK;
    do {
        if (h.flags & F_PREDICTOR) {
            if ((rc = ksc_predictor_weights(ix, nullptr, mlp_w.data()))) break;
            if ((rc = ksc_predictor_params(ix, &prm))) break;
        }
        if (h.flags & F_PRUNE_STATS) {
            cudaError_t e = cudaMalloc(&ix->pr_stats, s.pr_stats);
            if (e == cudaSuccess) e = cudaMalloc(&ix->pr_vecs, s.pr_vecs);
            if (e == cudaSuccess) e = cudaMemcpy(ix->pr_stats, pr_stats.data(), s.pr_stats, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(ix->pr_vecs, pr_vecs.data(), s.pr_vecs, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                set_error("loading the pruning statistics: %s", cudaGetErrorString(e));
                rc = e == cudaErrorMemoryAllocation ? KSC_ENOMEM : KSC_ECUDA;
                break;
            }
            ix->pr_have_stats = true;
        }
        if (h.flags & F_PRUNE_MODEL) {
            if ((rc = ksc_pruner_import_model(ix, pr_model.data()))) break;
            if (theta >= 0.f && (h.flags & F_PRUNE_STATS)) ix->pr_theta = theta;
        }
        if (h.flags & F_FILTER) {
            cudaError_t e = cudaMalloc(&ix->dims, s.dims);
            if (e == cudaSuccess) e = cudaMalloc(&ix->X_rr, s.X_full);
            if (e == cudaSuccess) e = cudaMemcpy(ix->dims, dims.data(), s.dims, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(ix->X_rr, X_full.data(), s.X_full, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                set_error("loading the component-filtration state: %s", cudaGetErrorString(e));
                rc = e == cudaErrorMemoryAllocation ? KSC_ENOMEM : KSC_ECUDA;
                break;
            }
            ix->h_dims = dims;
            ix->d_rr = h.d_full;
        }
    } while (0);
    if (rc != KSC_OK) {
        ksc_index_free(ix);
        return rc;
    }
    *out = ix;
    return KSC_OK;
}

}  // extern "C"
