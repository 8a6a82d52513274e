// Learned per-query nprobe / reorder (Sec. 4.2.1-4.2.2, Eq. 2): a small MLP
// stands in for the paper's gradient-boosted classifier.
//
// Features (F = 64) from the ranking step: the 32 smallest list distances
// d_1 <= ... <= d_32 (L2: ||q - c||^2; spherical: 1 - <q, c>) as d_i / mean(d)
// and the ratios d_1 / d_i.  Network F -> 64 -> 64 -> 2, ReLU, two sigmoid
// heads p_n (nprobe) and p_r (reorder), trained with binary cross-entropy on
// "hard query" labels that the plain search generates, by hand-written FP32
// forward / backward / Adam kernels.  Inference uses BF16-rounded weights and
// activations with FP32 accumulation, then Eq. 2 maps p to nprobe and R.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "index.cuh"
#include "mlp.cuh"

namespace ksc {

constexpr int MLP_TILE = 128;  // samples per CTA (training)
constexpr int MLP_ITILE = 32;  // queries per tile of the inference kernel (one warp's rows)

// Features of one query from its sorted ranking scores s[0..32).
__global__ void k_features(const float* __restrict__ scores, int64_t nq, int ld, int spherical,
                           float* __restrict__ feats) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const float* s = scores + q * ld;
    float mean = 0.f;
    for (int i = 0; i < MLP_FEAT_K; ++i) mean += fmaxf(feat_dist(s[i], spherical), 0.f);
    mean = mean / MLP_FEAT_K + 1e-12f;
    const float d1 = fmaxf(feat_dist(s[0], spherical), 0.f) + 1e-12f;
    float* f = feats + q * MLP_F;
    for (int i = 0; i < MLP_FEAT_K; ++i) {
        const float di = fmaxf(feat_dist(s[i], spherical), 0.f) + 1e-12f;
        f[i] = di / mean;
        f[MLP_FEAT_K + i] = d1 / di;
    }
}

// out[r][a] = act(sum_f in[r][f] W[a][f] + b[a]) for r < rows; W [A x Fin].
__device__ __forceinline__ void dense(const float* in, int rows, int Fin, const float* W, const float* b, int A,
                                      float* z, float* h) {
    for (int e = threadIdx.x; e < rows * A; e += blockDim.x) {
        const int r = e / A, a = e - r * A;
        float acc = b[a];
        for (int f = 0; f < Fin; ++f) acc = fmaf(in[r * Fin + f], W[a * Fin + f], acc);
        if (z) z[e] = acc;
        if (h) h[e] = acc > 0.f ? acc : 0.f;
    }
}

// One training pass over samples [0, B): loss (mean BCE over the batch, both
// heads) and gradients accumulated into grad (zeroed by the caller).  CTA c
// handles samples [c*128, c*128+128); the batch GEMMs run in shared memory.
// Network FN -> HN -> HN -> 2.
template <int FN, int HN>
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ w, const float* __restrict__ x,
                                                  const float* __restrict__ y, int64_t B, float* __restrict__ grad,
                                                  float* __restrict__ loss) {
    constexpr int NP = mlp_nparam<FN, HN>();
    extern __shared__ float sm[];
    float* sw = sm;                    // NP
    float* X = sw + NP;                // 128 x FN
    float* Z1 = X + MLP_TILE * FN;     // 128 x HN (pre-activation, then dZ1)
    float* Z2 = Z1 + MLP_TILE * HN;    // 128 x HN
    float* Hb = Z2 + MLP_TILE * HN;    // 128 x HN scratch (H1, then H2, then dH)
    float* D3 = Hb + MLP_TILE * HN;    // 128 x 2
    const int64_t r0 = (int64_t)blockIdx.x * MLP_TILE;
    const int rows = (int)(B - r0 < MLP_TILE ? B - r0 : MLP_TILE);
    for (int e = threadIdx.x; e < NP; e += blockDim.x) sw[e] = w[e];
    for (int e = threadIdx.x; e < rows * FN; e += blockDim.x) X[e] = x[r0 * FN + e];
    __syncthreads();
    const MlpW W = mlp_views_t<FN, HN>(sw);
    MlpW G = mlp_views_t<FN, HN>(grad);
    float* gW1 = const_cast<float*>(G.W1);
    float* gb1 = const_cast<float*>(G.b1);
    float* gW2 = const_cast<float*>(G.W2);
    float* gb2 = const_cast<float*>(G.b2);
    float* gW3 = const_cast<float*>(G.W3);
    float* gb3 = const_cast<float*>(G.b3);
    dense(X, rows, FN, W.W1, W.b1, HN, Z1, Hb);  // Hb = H1
    __syncthreads();
    dense(Hb, rows, HN, W.W2, W.b2, HN, Z2, nullptr);
    __syncthreads();
    // H2 overwrites H1 only after layer 2 consumed it
    for (int e = threadIdx.x; e < rows * HN; e += blockDim.x) Hb[e] = Z2[e] > 0.f ? Z2[e] : 0.f;
    __syncthreads();
    // output layer, loss and dZ3 = (p - y) / B
    float lsum = 0.f;
    for (int e = threadIdx.x; e < rows * MLP_O; e += blockDim.x) {
        const int r = e / MLP_O, o = e - r * MLP_O;
        float z = W.b3[o];
        for (int f = 0; f < HN; ++f) z = fmaf(Hb[r * HN + f], W.W3[o * HN + f], z);
        const float t = y[(r0 + r) * MLP_O + o];
        const float p = 1.f / (1.f + expf(-z));
        lsum += fmaxf(z, 0.f) - z * t + log1pf(expf(-fabsf(z)));
        D3[e] = (p - t) / (float)B;
    }
    __syncthreads();
    // gW3 = D3^T H2, gb3 = sum D3
    for (int e = threadIdx.x; e < MLP_O * HN; e += blockDim.x) {
        const int o = e / HN, f = e - o * HN;
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) acc = fmaf(D3[r * MLP_O + o], Hb[r * HN + f], acc);
        atomicAdd(&gW3[e], acc);
    }
    if (threadIdx.x < MLP_O) {
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) acc += D3[r * MLP_O + threadIdx.x];
        atomicAdd(&gb3[threadIdx.x], acc);
    }
    __syncthreads();
    // dZ2 = (D3 W3) * [Z2 > 0]  (into Z2)
    for (int e = threadIdx.x; e < rows * HN; e += blockDim.x) {
        const int r = e / HN, f = e - r * HN;
        float acc = 0.f;
        for (int o = 0; o < MLP_O; ++o) acc = fmaf(D3[r * MLP_O + o], W.W3[o * HN + f], acc);
        Z2[e] = Z2[e] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    // H1 again (layer 1 activations) for gW2
    for (int e = threadIdx.x; e < rows * HN; e += blockDim.x) Hb[e] = Z1[e] > 0.f ? Z1[e] : 0.f;
    __syncthreads();
    for (int e = threadIdx.x; e < HN * HN; e += blockDim.x) {
        const int a = e / HN, f = e - a * HN;
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) acc = fmaf(Z2[r * HN + a], Hb[r * HN + f], acc);
        atomicAdd(&gW2[e], acc);
    }
    for (int a = threadIdx.x; a < HN; a += blockDim.x) {
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) acc += Z2[r * HN + a];
        atomicAdd(&gb2[a], acc);
    }
    __syncthreads();
    // dZ1 = (dZ2 W2) * [Z1 > 0]  (into Z1)
    for (int e = threadIdx.x; e < rows * HN; e += blockDim.x) {
        const int r = e / HN, f = e - r * HN;
        float acc = 0.f;
        for (int a = 0; a < HN; ++a) acc = fmaf(Z2[r * HN + a], W.W2[a * HN + f], acc);
        Hb[e] = Z1[e] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < HN * FN; e += blockDim.x) {
        const int a = e / FN, f = e - a * FN;
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) acc = fmaf(Hb[r * HN + a], X[r * FN + f], acc);
        atomicAdd(&gW1[e], acc);
    }
    for (int a = threadIdx.x; a < HN; a += blockDim.x) {
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) acc += Hb[r * HN + a];
        atomicAdd(&gb1[a], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, lsum / (float)B);
}

// Adam (Kingma & Ba 2015), bias-corrected, on every parameter.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// One layer for a tile of rows: thread e computes unit a = e / rows of row
// r = e % rows, so a warp shares one weight row (broadcast) and reads 32
// activation rows of stride MLP_LDI (odd: distinct banks).  Accumulation in
// ascending input order, as in dense().
constexpr int MLP_LDI = MLP_F + 1;  // (MLP_F == MLP_H)
__device__ __forceinline__ void dense_rows(const float* in, int rows, int Fin, const float* W, const float* b, int A,
                                           float* out, bool relu_bf) {
    for (int e = threadIdx.x; e < rows * A; e += blockDim.x) {
        const int a = e / rows, r = e - a * rows;
        float acc = b[a];
        for (int f = 0; f < Fin; ++f) acc = fmaf(in[r * MLP_LDI + f], W[a * Fin + f], acc);
        out[r * MLP_LDI + a] = relu_bf ? bf(acc > 0.f ? acc : 0.f) : acc;
    }
}

// Inference: BF16 weights and activations, FP32 accumulation; probabilities
// and the Eq. 2 parameters per query.  Persistent CTAs over tiles of
// MLP_ITILE queries.
__global__ void __launch_bounds__(256) k_mlp_infer(const float* __restrict__ w, const float* __restrict__ x,
                                                   int64_t B, ksc_adaptive_params prm, float* __restrict__ prob,
                                                   int32_t* __restrict__ nprobe, int32_t* __restrict__ rerank) {
    extern __shared__ float sm[];
    float* sw = sm;
    float* X = sw + MLP_NPARAM;
    float* H1 = X + MLP_ITILE * MLP_LDI;
    float* H2 = H1 + MLP_ITILE * MLP_LDI;
    for (int e = threadIdx.x; e < MLP_NPARAM; e += blockDim.x) sw[e] = bf(w[e]);
    const MlpW W = mlp_views(sw);
    for (int64_t r0 = (int64_t)blockIdx.x * MLP_ITILE; r0 < B; r0 += (int64_t)gridDim.x * MLP_ITILE) {
        const int rows = (int)(B - r0 < MLP_ITILE ? B - r0 : MLP_ITILE);
        for (int e = threadIdx.x; e < rows * MLP_F; e += blockDim.x) {
            const int r = e / MLP_F, f = e - r * MLP_F;
            X[r * MLP_LDI + f] = bf(x[(r0 + r) * MLP_F + f]);
        }
        __syncthreads();
        dense_rows(X, rows, MLP_F, W.W1, W.b1, MLP_H, H1, true);
        __syncthreads();
        dense_rows(H1, rows, MLP_H, W.W2, W.b2, MLP_H, H2, true);
        __syncthreads();
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
            float p[MLP_O];
            for (int o = 0; o < MLP_O; ++o) {
                float z = W.b3[o];
                for (int f = 0; f < MLP_H; ++f) z = fmaf(H2[r * MLP_LDI + f], W.W3[o * MLP_H + f], z);
                p[o] = 1.f / (1.f + expf(-z));
                if (prob) prob[(r0 + r) * MLP_O + o] = p[o];
            }
            if (nprobe)
                nprobe[r0 + r] = prm.regression ? regmap(p[0], prm.pmin, prm.pmax, prm.p0, prm.p1)
                                                : eq2(p[0], prm.pmin, prm.pmax, prm.p0, prm.p1);
            if (rerank)
                rerank[r0 + r] = prm.regression ? regmap(p[1], prm.rmin, prm.rmax, prm.r0, prm.r1)
                                                : eq2(p[1], prm.rmin, prm.rmax, prm.r0, prm.r1);
        }
        __syncthreads();  // the tile buffers are reused
    }
}

// The adaptive search's head in one kernel: per tile of 32 RPT queries the
// features of each query from its sorted ranking distances (as k_features),
// then the network and the settings (as k_mlp_infer).  Each output unit is
// accumulated in the same order from the same BF16-rounded operands as
// there, so the settings are bit for bit those of the two kernels; what
// differs is the blocking: the weights are staged transposed ([f][a]) and
// the activations feature-major ([f][r]), and each of the 512 threads keeps a
// block of 4 units x RPT rows in registers (a warp: one group of 4 units for
// all rows of the tile), so that RPT activations and a float4 of weights (a
// broadcast) feed 4 RPT FMAs.  The weight loads are issued first and stored
// after the features, so that their latency overlaps the feature loads.
constexpr int MLP_STHREADS = 512;  // threads per CTA: 32 row groups x MLP_H / 4 unit groups
constexpr int MLP_SLD = 68;        // row stride of the transposed weights (16-byte aligned, staggered banks)
constexpr int MLP_SW = MLP_F * MLP_SLD;
static_assert(MLP_F == 64 && MLP_H == 64 && MLP_O == 2 && MLP_FEAT_K * 2 == MLP_F, "head layout");
static_assert(MLP_STHREADS == 32 * (MLP_H / 4), "one block of 4 units per thread");
template <int RPT>
constexpr int mlp_xld() { return 32 * RPT + 4; }  // row stride of the activations
template <int RPT>
constexpr size_t mlp_scores_smem() {
    return sizeof(float) * (2 * MLP_SW + 2 * MLP_F * mlp_xld<RPT>() + 2 * MLP_H + MLP_O * MLP_H + 4);
}

// HT[a][r] = bf(relu(b[a] + sum_f XT[f][r] WT[f][a])) for the thread's block
// (units 4 ug.., rows rg + 32 t for t < RPT: a warp's loads of one row index
// are consecutive words, conflict-free).
template <int RPT>
__device__ __forceinline__ void dense_block(const float* XT, const float* WT, const float* bsm, float* HT, int rg,
                                           int ug) {
    constexpr int XLD = mlp_xld<RPT>();
    float acc[4][RPT];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int t = 0; t < RPT; ++t) acc[j][t] = bsm[4 * ug + j];
#pragma unroll 8
    for (int f = 0; f < MLP_F; ++f) {
        float x[RPT];
#pragma unroll
        for (int t = 0; t < RPT; ++t) x[t] = XT[f * XLD + rg + 32 * t];
        const float4 wv = *reinterpret_cast<const float4*>(WT + f * MLP_SLD + 4 * ug);
        const float ws[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int t = 0; t < RPT; ++t) acc[j][t] = fmaf(x[t], ws[j], acc[j][t]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int t = 0; t < RPT; ++t) HT[(4 * ug + j) * XLD + rg + 32 * t] = bf(acc[j][t] > 0.f ? acc[j][t] : 0.f);
}

template <int RPT>
__global__ void __launch_bounds__(MLP_STHREADS) k_mlp_infer_scores(const float* __restrict__ scores, int ld,
                                                                   int spherical, const float* __restrict__ w,
                                                                   int64_t B, ksc_adaptive_params prm,
                                                                   int32_t* __restrict__ nprobe,
                                                                   int32_t* __restrict__ rerank) {
    constexpr int TILE = 32 * RPT, XLD = mlp_xld<RPT>();
    extern __shared__ float4 msm4[];
    __shared__ float s_mean[TILE], s_d1[TILE];
    float* WT1 = reinterpret_cast<float*>(msm4);
    float* WT2 = WT1 + MLP_SW;
    float* XT = WT2 + MLP_SW;       // features (first the clamped distances), then the second hidden layer
    float* HT = XT + MLP_F * XLD;   // first hidden layer
    float* b1 = HT + MLP_F * XLD;
    float* b2 = b1 + MLP_H;
    float* W3 = b2 + MLP_H;
    float* b3 = W3 + MLP_O * MLP_H;
    const MlpW G = mlp_views(w);
    // both hidden matrices in one round of 16-byte loads; thread t takes row
    // a = t % 64 of each (so that the transposed stores of a warp fall in
    // distinct banks)
    constexpr int V = MLP_H * MLP_F / 4 / MLP_STHREADS;
    float4 v1[V], v2[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
        const int a = threadIdx.x & (MLP_H - 1), fq = (threadIdx.x >> 6) + (MLP_STHREADS / MLP_H) * u;
        v1[u] = __ldg(reinterpret_cast<const float4*>(G.W1 + a * MLP_F) + fq);
        v2[u] = __ldg(reinterpret_cast<const float4*>(G.W2 + a * MLP_H) + fq);  // (MLP_F == MLP_H)
    }
    const int rg = threadIdx.x & 31, ug = threadIdx.x >> 5;
    bool staged = false;
    for (int64_t r0 = (int64_t)blockIdx.x * TILE; r0 < B; r0 += (int64_t)gridDim.x * TILE) {
        const int rows = (int)(B - r0 < TILE ? B - r0 : TILE);
        // the clamped distances u_i = max(dist_i, 0) of every row (XT's first
        // FEAT_K rows), then per row the mean in ascending order by one thread
        for (int e = threadIdx.x; e < TILE * MLP_FEAT_K; e += blockDim.x) {
            const int r = e % TILE, i = e / TILE;
            XT[i * XLD + r] = r < rows ? fmaxf(feat_dist(__ldg(scores + (r0 + r) * ld + i), spherical), 0.f) : 0.f;
        }
        if (!staged) {
#pragma unroll
            for (int u = 0; u < V; ++u) {
                const int a = threadIdx.x & (MLP_H - 1), f = 4 * ((threadIdx.x >> 6) + (MLP_STHREADS / MLP_H) * u);
                WT1[f * MLP_SLD + a] = bf(v1[u].x);
                WT1[(f + 1) * MLP_SLD + a] = bf(v1[u].y);
                WT1[(f + 2) * MLP_SLD + a] = bf(v1[u].z);
                WT1[(f + 3) * MLP_SLD + a] = bf(v1[u].w);
                WT2[f * MLP_SLD + a] = bf(v2[u].x);
                WT2[(f + 1) * MLP_SLD + a] = bf(v2[u].y);
                WT2[(f + 2) * MLP_SLD + a] = bf(v2[u].z);
                WT2[(f + 3) * MLP_SLD + a] = bf(v2[u].w);
            }
            if (threadIdx.x < MLP_H) {
                b1[threadIdx.x] = bf(G.b1[threadIdx.x]);
                b2[threadIdx.x] = bf(G.b2[threadIdx.x]);
            }
            if (threadIdx.x < MLP_O * MLP_H) W3[threadIdx.x] = bf(G.W3[threadIdx.x]);
            if (threadIdx.x < MLP_O) b3[threadIdx.x] = bf(G.b3[threadIdx.x]);
            staged = true;
        }
        __syncthreads();
        if (threadIdx.x < TILE) {
            float mean = 0.f;
#pragma unroll
            for (int i = 0; i < MLP_FEAT_K; ++i) mean += XT[i * XLD + threadIdx.x];
            s_mean[threadIdx.x] = mean / MLP_FEAT_K + 1e-12f;
            s_d1[threadIdx.x] = XT[threadIdx.x] + 1e-12f;
        }
        __syncthreads();
        // features: u_i / mean and d_1 / u_i (+ 1e-12 each), rounded to BF16;
        // the second half first, since the first overwrites the u_i
        for (int e = threadIdx.x; e < TILE * MLP_FEAT_K; e += blockDim.x) {
            const int r = e % TILE, i = e / TILE;
            const float di = XT[i * XLD + r] + 1e-12f;
            const bool in = r < rows;
            XT[(MLP_FEAT_K + i) * XLD + r] = in ? bf(s_d1[r] / di) : 0.f;
            XT[i * XLD + r] = in ? bf(di / s_mean[r]) : 0.f;
        }
        __syncthreads();
        dense_block<RPT>(XT, WT1, b1, HT, rg, ug);
        __syncthreads();
        dense_block<RPT>(HT, WT2, b2, XT, rg, ug);
        __syncthreads();
        if (threadIdx.x < MLP_O * TILE) {
            const int r = threadIdx.x % TILE, o = threadIdx.x / TILE;
            if (r < rows) {
                float z = b3[o];
                for (int f = 0; f < MLP_H; ++f) z = fmaf(XT[f * XLD + r], W3[o * MLP_H + f], z);
                const float p = 1.f / (1.f + expf(-z));
                if (o == 0)
                    nprobe[r0 + r] = prm.regression ? regmap(p, prm.pmin, prm.pmax, prm.p0, prm.p1)
                                                    : eq2(p, prm.pmin, prm.pmax, prm.p0, prm.p1);
                else
                    rerank[r0 + r] = prm.regression ? regmap(p, prm.rmin, prm.rmax, prm.r0, prm.r1)
                                                    : eq2(p, prm.rmin, prm.rmax, prm.r0, prm.r1);
            }
        }
        __syncthreads();  // XT, s_mean and s_d1 are reused by the next tile
    }
}

// Hits of a search result: how many of the k returned distances are at most
// the query's true k-th distance (ties count), for the label rule.
__global__ void k_hits(const float* __restrict__ dists, int64_t nq, int k, const float* __restrict__ kth, int ip,
                       int32_t* __restrict__ hits) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const float t = kth[q];
    const float tol = 1e-5f * fabsf(t) + 1e-6f;
    int h = 0;
    for (int r = 0; r < k; ++r) {
        const float dv = dists[q * k + r];
        h += ip ? (dv >= t - tol) : (dv <= t + tol);
    }
    hits[q] = h;
}

template <int F, int H>
static size_t grad_smem() {
    return sizeof(float) * (mlp_nparam<F, H>() + MLP_TILE * (F + 3 * H + MLP_O));
}
static size_t infer_smem() { return sizeof(float) * (MLP_NPARAM + 3 * MLP_ITILE * MLP_LDI); }

template <int F, int H>
static int mlp_grad_t(const float* w, const float* x, const float* y, int64_t B, float* grad, float* loss,
                      cudaStream_t st) {
    KSC_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * mlp_nparam<F, H>(), st));
    if (loss) KSC_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st));
    KSC_CUDA(cudaFuncSetAttribute(k_mlp_grad<F, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)grad_smem<F, H>()));
    k_mlp_grad<F, H><<<(unsigned)((B + MLP_TILE - 1) / MLP_TILE), 256, grad_smem<F, H>(), st>>>(w, x, y, B, grad,
                                                                                              loss);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

int mlp_grad(const float* w, const float* x, const float* y, int64_t B, float* grad, float* loss, cudaStream_t st) {
    return mlp_grad_t<MLP_F, MLP_H>(w, x, y, B, grad, loss, st);
}

// The pruning classifier's network (Sec. 4.2.3): 16 -> 32 -> 32 -> 2.
int prune_mlp_grad(const float* w, const float* x, const float* y, int64_t B, float* grad, float* loss,
                   cudaStream_t st) {
    static_assert(mlp_nparam<KSC_PRUNE_FEATURES, 32>() == KSC_PRUNE_NPARAMS, "pruning network size");
    return mlp_grad_t<KSC_PRUNE_FEATURES, 32>(w, x, y, B, grad, loss, st);
}

int mlp_infer(const float* w, const float* x, int64_t B, const ksc_adaptive_params& prm, float* prob,
              int32_t* nprobe, int32_t* rerank, cudaStream_t st) {
    KSC_CUDA(cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)infer_smem()));
    // persistent over row tiles: the weights are staged once per CTA
    int per_sm = 0;
    KSC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_infer, 256, infer_smem()));
    const int64_t tiles = (B + MLP_ITILE - 1) / MLP_ITILE;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1));
    k_mlp_infer<<<(unsigned)(grid > 0 ? grid : 1), 256, infer_smem(), st>>>(w, x, B, prm, prob, nprobe, rerank);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

int mlp_infer_scores(const float* w, const float* scores, int ld, int spherical, int64_t B,
                     const ksc_adaptive_params& prm, int32_t* nprobe, int32_t* rerank, cudaStream_t st) {
    if (B == 0) return KSC_OK;
    // tiles of 64 queries, or of 96 when that keeps to one CTA per SM
    const int64_t sms = num_sms();
    if ((B + 63) / 64 <= sms || (B + 95) / 96 > sms) {
        KSC_CUDA(cudaFuncSetAttribute(k_mlp_infer_scores<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)mlp_scores_smem<2>()));
        const int64_t grid = std::min<int64_t>((B + 63) / 64, sms * 2);
        k_mlp_infer_scores<2><<<(unsigned)grid, MLP_STHREADS, mlp_scores_smem<2>(), st>>>(scores, ld, spherical, w,
                                                                                          B, prm, nprobe, rerank);
    } else {
        KSC_CUDA(cudaFuncSetAttribute(k_mlp_infer_scores<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)mlp_scores_smem<3>()));
        k_mlp_infer_scores<3><<<(unsigned)((B + 95) / 96), MLP_STHREADS, mlp_scores_smem<3>(), st>>>(
            scores, ld, spherical, w, B, prm, nprobe, rerank);
    }
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

int mlp_features(const float* scores, int64_t nq, int ld, int spherical, float* feats, cudaStream_t st) {
    k_features<<<(unsigned)((nq + 127) / 128), 128, 0, st>>>(scores, nq, ld, spherical, feats);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

int mlp_hits(const float* dists, int64_t nq, int k, const float* kth, int ip, int32_t* hits, cudaStream_t st) {
    k_hits<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(dists, nq, k, kth, ip, hits);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

int mlp_adam_n(float* w, const float* g, float* m, float* v, int n, int t, float lr, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
    k_adam<<<(n + 255) / 256, 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, 1e-8f, bc1, bc2);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

int mlp_adam(float* w, const float* g, float* m, float* v, int t, float lr, cudaStream_t st) {
    return mlp_adam_n(w, g, m, v, MLP_NPARAM, t, lr, st);
}

}  // namespace ksc
