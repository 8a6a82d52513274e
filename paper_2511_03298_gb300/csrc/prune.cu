// Predictive cluster pruning (Sec. 4.2.3, Table 4; Alg. 2 f_prune).
//
// A classifier per (query, probed list) predicts whether the list holds one of
// the query's true nearest neighbours; lists it rejects are dropped from the
// query's probe list before the work lists are built, so the scan itself runs
// unchanged (no divergence in it).  The features of Table 4 come from per-list
// statistics computed once (size, radius, distance moments and histogram,
// outliers and their mean offset, two principal axes) and a few dot products
// with the query; the classifier is an MLP 16 -> 32 -> 32 -> 2 (head 0 used)
// trained by the FP32 kernels of mlp.cu.
#include <algorithm>
#include <cmath>

#include "index.cuh"

namespace ksc {

constexpr int PR_NSTAT = KSC_PRUNE_STATS;
constexpr int PR_NF = KSC_PRUNE_FEATURES;
constexpr int PR_H = 32;
constexpr int PR_NP = KSC_PRUNE_NPARAMS;
constexpr int PR_WARPS = 8;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA of one double per thread, in a fixed order (deterministic);
// every thread gets the total.  red: PR_WARPS doubles of shared memory.
__device__ double block_sum_d(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();  // red is free
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < PR_WARPS; ++w) s += red[w];
    return s;
}

// ------------------------------------------------------------------ list statistics
// One CTA per list p (members = the first n_p slots of the list's blocks).
// A warp takes members m = warp, warp + 8, ... in order, a lane holds the
// offset dims t = lane + 32 i (i < DPL) in registers; per-warp partial
// vectors are summed over the warps in a fixed order, so the result does not
// depend on scheduling.  Distances in FP32, moments accumulated in FP64.
// Shared memory: c, v1, v2, w (d each) and PR_WARPS x d partials.
template <int DPL>
__global__ void __launch_bounds__(PR_WARPS * 32) k_prune_stats(const float* __restrict__ X, int d,
                                                               const float* __restrict__ c_mean,
                                                               const int64_t* __restrict__ boff,
                                                               const int32_t* __restrict__ list_n,
                                                               const int32_t* __restrict__ blk_ids, int iters,
                                                               float* __restrict__ dscr, float* __restrict__ stats,
                                                               float* __restrict__ vecs) {
    extern __shared__ float psm[];
    float* c = psm;
    float* v1 = c + d;
    float* v2 = v1 + d;
    float* w = v2 + d;
    float* part = w + d;  // PR_WARPS x d
    __shared__ double red[PR_WARPS];
    __shared__ double s_mu, s_sig;
    __shared__ int s_hist[4], s_nout;
    const int p = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = list_n[p];
    float* st = stats + (int64_t)p * PR_NSTAT;
    float* vv = vecs + (int64_t)p * 3 * d;
    if (n == 0) {
        for (int e = threadIdx.x; e < PR_NSTAT; e += blockDim.x) st[e] = 0.f;
        for (int e = threadIdx.x; e < 3 * d; e += blockDim.x) vv[e] = 0.f;
        return;
    }
    const int64_t base = boff[p] * 32;
    for (int t = threadIdx.x; t < d; t += blockDim.x) c[t] = c_mean[(int64_t)p * d + t];
    if (threadIdx.x < 4) s_hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_nout = 0;
    __syncthreads();
    auto load_r = [&](int m, float (&r)[DPL]) {
        const float* x = X + (int64_t)blk_ids[base + m] * d;
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
            const int t = lane + 32 * i;
            r[i] = t < d ? __fsub_rn(x[t], c[t]) : 0.f;
        }
    };
    // 1. distances |r|, radius and mean
    float rmax = 0.f;
    double dsum = 0.0;
    for (int m = warp; m < n; m += PR_WARPS) {
        float r[DPL];
        load_r(m, r);
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) s = fmaf(r[i], r[i], s);
        const float dist = sqrtf(warp_sum_f(s));
        if (lane == 0) {
            dscr[base + m] = dist;
            rmax = fmaxf(rmax, dist);
            dsum += dist;
        }
    }
    // radius: max over the lane-0 values (exact in any order)
    __shared__ float s_rmax[PR_WARPS];
    if (lane == 0) s_rmax[warp] = rmax;
    const double tot = block_sum_d(lane == 0 ? dsum : 0.0, red);
    float rho = 0.f;
    for (int i = 0; i < PR_WARPS; ++i) rho = fmaxf(rho, s_rmax[i]);
    if (threadIdx.x == 0) s_mu = tot / n;
    __syncthreads();
    const double mu = s_mu;
    // 2. std, histogram, outliers (thread per member)
    double vs = 0.0;
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
        const float dist = dscr[base + m];
        vs += ((double)dist - mu) * ((double)dist - mu);
    }
    const double var = block_sum_d(vs, red);
    if (threadIdx.x == 0) s_sig = sqrt(var / n);
    __syncthreads();
    const double sig = s_sig, thr = mu + 2.0 * sig;
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
        const float dist = dscr[base + m];
        const int b = dist > 0.75f * rho ? 3 : (dist > 0.5f * rho ? 2 : (dist > 0.25f * rho ? 1 : 0));
        atomicAdd(&s_hist[b], 1);
        if ((double)dist > thr) atomicAdd(&s_nout, 1);
    }
    // 3. mean outlier offset
    float acc[DPL];
#pragma unroll
    for (int i = 0; i < DPL; ++i) acc[i] = 0.f;
    for (int m = warp; m < n; m += PR_WARPS) {
        if (!((double)dscr[base + m] > thr)) continue;
        float r[DPL];
        load_r(m, r);
#pragma unroll
        for (int i = 0; i < DPL; ++i) acc[i] += r[i];
    }
    auto combine = [&](float (&a)[DPL]) {  // w = sum over warps of a, fixed order
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
            const int t = lane + 32 * i;
            if (t < d) part[warp * d + t] = a[i];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < d; t += blockDim.x) {
            float s = 0.f;
            for (int q = 0; q < PR_WARPS; ++q) s += part[q * d + t];
            w[t] = s;
        }
        __syncthreads();
    };
    combine(acc);
    const int nout = s_nout;
    for (int t = threadIdx.x; t < d; t += blockDim.x) vv[2 * d + t] = nout > 0 ? w[t] / (float)nout : 0.f;
    // 4. principal axes by power iterations: w = sum_m <r_m, v> r_m
    auto power_step = [&](const float* v) {
        float a[DPL];
#pragma unroll
        for (int i = 0; i < DPL; ++i) a[i] = 0.f;
        for (int m = warp; m < n; m += PR_WARPS) {
            float r[DPL];
            load_r(m, r);
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < DPL; ++i) {
                const int t = lane + 32 * i;
                if (t < d) s = fmaf(r[i], v[t], s);
            }
            s = warp_sum_f(s);
#pragma unroll
            for (int i = 0; i < DPL; ++i) a[i] = fmaf(s, r[i], a[i]);
        }
        combine(a);
    };
    // v <- w / |w| (v kept when w = 0); optionally with `proj` projected out of w first
    auto normalise = [&](float* v, const float* proj) {
        if (proj) {
            double pp = 0.0;
            for (int t = threadIdx.x; t < d; t += blockDim.x) pp += (double)w[t] * proj[t];
            const float a = (float)block_sum_d(pp, red);
            for (int t = threadIdx.x; t < d; t += blockDim.x) w[t] = fmaf(-a, proj[t], w[t]);
            __syncthreads();
        }
        double nn = 0.0;
        for (int t = threadIdx.x; t < d; t += blockDim.x) nn += (double)w[t] * w[t];
        const double tn = block_sum_d(nn, red);
        if (tn > 0.0) {
            const float inv = (float)(1.0 / sqrt(tn));
            for (int t = threadIdx.x; t < d; t += blockDim.x) v[t] = w[t] * inv;
        }
        __syncthreads();
    };
    const float s0 = (float)(1.0 / sqrt((double)d));
    for (int t = threadIdx.x; t < d; t += blockDim.x) v1[t] = s0;
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
        power_step(v1);
        normalise(v1, nullptr);
    }
    for (int t = threadIdx.x; t < d; t += blockDim.x) w[t] = (t & 1) ? -s0 : s0;
    __syncthreads();
    normalise(v2, v1);
    for (int it = 0; it < iters; ++it) {
        power_step(v2);
        normalise(v2, v1);
    }
    // 5. variances along the axes
    double l1 = 0.0, l2 = 0.0;
    for (int m = warp; m < n; m += PR_WARPS) {
        float r[DPL];
        load_r(m, r);
        float a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
            const int t = lane + 32 * i;
            if (t < d) {
                a1 = fmaf(r[i], v1[t], a1);
                a2 = fmaf(r[i], v2[t], a2);
            }
        }
        a1 = warp_sum_f(a1);
        a2 = warp_sum_f(a2);
        if (lane == 0) {
            l1 += (double)a1 * a1;
            l2 += (double)a2 * a2;
        }
    }
    const double L1 = block_sum_d(lane == 0 ? l1 : 0.0, red);
    const double L2 = block_sum_d(lane == 0 ? l2 : 0.0, red);
    for (int t = threadIdx.x; t < d; t += blockDim.x) {
        vv[t] = v1[t];
        vv[d + t] = v2[t];
    }
    if (threadIdx.x == 0) {
        st[0] = (float)n;
        st[1] = rho;
        st[2] = (float)mu;
        st[3] = (float)sig;
        for (int b = 0; b < 4; ++b) st[4 + b] = (float)s_hist[b] / (float)n;
        st[8] = (float)nout / (float)n;
        st[9] = (float)(L1 / n);
        st[10] = (float)(L2 / n);
        st[11] = 0.f;
    }
}

int prune_stats(ksc_index* ix, int iters, cudaStream_t st) {
    KSC_CHECK_ARG(ix->d <= 1024, "pruning statistics need d <= 1024");
    if (iters <= 0) iters = 30;
    if (!ix->pr_stats) KSC_CUDA(cudaMalloc(&ix->pr_stats, sizeof(float) * ix->L * PR_NSTAT));
    if (!ix->pr_vecs) KSC_CUDA(cudaMalloc(&ix->pr_vecs, sizeof(float) * ix->L * 3 * ix->d));
    bump_workspace_generation();
    float* dscr = nullptr;
    KSC_CUDA(cudaMalloc(&dscr, sizeof(float) * ix->nblocks * 32 + 16));
    const size_t smem = sizeof(float) * (size_t)(4 + PR_WARPS) * ix->d;
    int rc = KSC_OK;
#define KSC_PS(DPL)                                                                                              \
    do {                                                                                                         \
        cudaFuncSetAttribute(k_prune_stats<DPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
        k_prune_stats<DPL><<<ix->L, PR_WARPS * 32, smem, st>>>(ix->X, ix->d, ix->c_mean, ix->list_boff,          \
                                                               ix->list_n, ix->blk_ids, iters, dscr,             \
                                                               ix->pr_stats, ix->pr_vecs);                       \
    } while (0)
    if (ix->d <= 128) KSC_PS(4);
    else if (ix->d <= 256) KSC_PS(8);
    else if (ix->d <= 512) KSC_PS(16);
    else KSC_PS(32);
#undef KSC_PS
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("k_prune_stats: %s", cudaGetErrorString(e));
        rc = KSC_ECUDA;
    }
    cudaStreamSynchronize(st);  // the scratch is freed below
    cudaFree(dscr);
    if (rc == KSC_OK) ix->pr_have_stats = true;
    return rc;
}

// ------------------------------------------------------------------ rows (q, r)
struct PruneArgs {
    const float* Q;
    int64_t nq;
    int d, L;
    const float* c_mean;
    const int32_t* probes;
    int Pmax;
    const int32_t* nprobe;
    int P;
    const float* stats;
    const float* vecs;
    const float* model;  // KSC_PRUNE_MODEL floats, or null (features only)
    float theta;
    float* feats;
    float* prob;
    int32_t* probes_out;
    int32_t* nprobe_out;
};

// Persistent CTAs (the model staged once per CTA in shared memory), each
// taking groups of QB = 256 / Pmax queries, i.e. up to 256 (query, rank) rows:
//  1. a warp per query forms the dot products of its rows over d with the
//     lanes across d (coalesced; two rows per step, so their loads overlap):
//     |q - c_p|^2, |q - c_{rank 0}|^2, <v1, q - c_p>, <v2, q - c_p>,
//     <outlier offset, q - c_p>, kept in shared memory per row;
//  2. a thread per row turns them into its 16 features and runs the MLP (all
//     threads read the same weight at a time: a shared-memory broadcast).
// Rows r >= P_q are skipped.  Keep probability into prob, features into feats.
constexpr int PR_ROWS = 256;  // rows per group = threads per CTA

template <int DPL>
__global__ void __launch_bounds__(PR_ROWS, 2) k_prune_rows(PruneArgs A) {
    __shared__ __align__(16) float sm[KSC_PRUNE_MODEL];
    __shared__ float sx[PR_NF][PR_ROWS];  // each row's standardised features
    __shared__ float sdot[5][PR_ROWS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (A.model) {
        for (int e = threadIdx.x; e < KSC_PRUNE_MODEL; e += blockDim.x) sm[e] = A.model[e];
        __syncthreads();
        if (threadIdx.x < PR_NF) sm[PR_NP + PR_NF + threadIdx.x] = 1.f / sm[PR_NP + PR_NF + threadIdx.x];
    }
    __syncthreads();
    const float* W1 = sm;
    const float* b1 = W1 + PR_H * PR_NF;
    const float* W2 = b1 + PR_H;
    const float* b2 = W2 + PR_H * PR_H;
    const float* W3 = b2 + PR_H;  // row 0 = head 0
    const float* mu = sm + PR_NP;
    const float* inv = mu + PR_NF;  // 1 / std
    const int d = A.d, Pmax = A.Pmax;
    const int QB = PR_ROWS / Pmax;  // >= 1 (Pmax <= PR_ROWS)
    const int64_t ngroups = (A.nq + QB - 1) / QB;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int64_t q0 = grp * QB;
        // 1. dot products, a warp per query
        for (int qi = warp; qi < QB; qi += PR_ROWS / 32) {
            const int64_t q = q0 + qi;
            if (q >= A.nq) break;
            int Pq = A.nprobe ? A.nprobe[q] : A.P;
            Pq = Pq < 1 ? 1 : (Pq > Pmax ? Pmax : Pq);
            const int32_t* pr = A.probes + q * Pmax;
            const int p0 = pr[0];
            const bool ok0 = p0 >= 0 && p0 < A.L;
            float qv[DPL], e0s = 0.f;
#pragma unroll
            for (int i = 0; i < DPL; ++i) {
                const int t = lane + 32 * i;
                qv[i] = t < d ? A.Q[q * d + t] : 0.f;
                if (t < d && ok0) {
                    const float e0 = __fsub_rn(qv[i], A.c_mean[(int64_t)p0 * d + t]);
                    e0s = fmaf(e0, e0, e0s);
                }
            }
            e0s = warp_sum_f(e0s);
            for (int r = 0; r < Pq; r += 2) {
                float v[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int rr = r + h;
                    const int p = rr < Pq ? pr[rr] : -1;
                    if (p < 0 || p >= A.L) continue;
                    const float* cp = A.c_mean + (int64_t)p * d;
                    const float* vp = A.vecs + (int64_t)p * 3 * d;
#pragma unroll
                    for (int i = 0; i < DPL; ++i) {
                        const int t = lane + 32 * i;
                        if (t < d) {
                            const float e = __fsub_rn(qv[i], cp[t]);
                            v[h][0] = fmaf(e, e, v[h][0]);
                            v[h][1] = fmaf(vp[t], e, v[h][1]);
                            v[h][2] = fmaf(vp[d + t], e, v[h][2]);
                            v[h][3] = fmaf(vp[2 * d + t], e, v[h][3]);
                        }
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int c = 0; c < 4; ++c) v[h][c] = warp_sum_f(v[h][c]);
                if (lane == 0) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (r + h >= Pq) break;
                        const int row = qi * Pmax + r + h;
                        sdot[0][row] = v[h][0];
                        sdot[1][row] = e0s;
                        sdot[2][row] = v[h][1];
                        sdot[3][row] = v[h][2];
                        sdot[4][row] = v[h][3];
                    }
                }
            }
        }
        __syncthreads();
        // 2. features and the MLP, a thread per row
        const int t = threadIdx.x;
        const int qi = t / Pmax, r = t - qi * Pmax;
        const int64_t q = q0 + qi;
        if (qi < QB && q < A.nq) {
            int Pq = A.nprobe ? A.nprobe[q] : A.P;
            Pq = Pq < 1 ? 1 : (Pq > Pmax ? Pmax : Pq);
            const int64_t row = q * Pmax + r;
            float f[PR_NF];
#pragma unroll
            for (int e = 0; e < PR_NF; ++e) f[e] = 0.f;
            const int32_t* pr = A.probes + q * Pmax;
            const int p = r < Pq ? pr[r] : -1, p0 = pr[0];
            if (p >= 0 && p < A.L) {
                const bool ok0 = p0 >= 0 && p0 < A.L;
                const float* stp = A.stats + (int64_t)p * PR_NSTAT;
                const float D0 = ok0 ? sqrtf(sdot[1][t]) : 0.f;
                const float rho0 = ok0 ? A.stats[(int64_t)p0 * PR_NSTAT + 1] : 0.f;
                const float ig = 1.f / fmaxf(D0, 1e-9f);
                const float D = sqrtf(sdot[0][t]), iD = 1.f / fmaxf(D, 1e-9f), rho = stp[1];
                const float u1 = sdot[2][t] * iD * ig, u2 = sdot[3][t] * iD * ig;
                f[0] = D / fmaxf(rho, 1e-9f);
                f[1] = D * ig;
                f[2] = (D - rho) * ig;
                f[3] = __logf(1.f + stp[0]);
                f[4] = rho * ig;
                f[5] = stp[2] * ig;
                f[6] = stp[3] * ig;
                f[7] = stp[4];
                f[8] = stp[5];
                f[9] = stp[6];
                f[10] = stp[7];
                f[11] = stp[8];
                f[12] = stp[9] * u1 * u1;
                f[13] = stp[10] * u2 * u2;
                f[14] = sdot[4][t] * iD * ig;
                f[15] = D0 / fmaxf(rho0, 1e-9f);
            }
            if (A.feats) {
#pragma unroll
                for (int e = 0; e < PR_NF; e += 4)
                    *reinterpret_cast<float4*>(A.feats + row * PR_NF + e) = make_float4(f[e], f[e + 1], f[e + 2], f[e + 3]);
            }
            if (A.model && r < Pq) {
#pragma unroll
                for (int e = 0; e < PR_NF; ++e) sx[e][t] = (f[e] - mu[e]) * inv[e];
                // layer 1 input by input (ascending), all 32 units in registers
                float h1[PR_H];
#pragma unroll
                for (int a = 0; a < PR_H; ++a) h1[a] = b1[a];
#pragma unroll 1
                for (int e = 0; e < PR_NF; ++e) {
                    const float x = sx[e][t];
#pragma unroll
                    for (int a = 0; a < PR_H; ++a) h1[a] = fmaf(x, W1[a * PR_NF + e], h1[a]);
                }
                float zz = W3[2 * PR_H];
#pragma unroll 1
                for (int a = 0; a < PR_H; ++a) {
                    float acc = b2[a];
#pragma unroll
                    for (int e = 0; e < PR_H; ++e) acc = fmaf(fmaxf(h1[e], 0.f), W2[a * PR_H + e], acc);
                    zz = fmaf(fmaxf(acc, 0.f), W3[a], zz);
                }
                A.prob[row] = 1.f / (1.f + __expf(-zz));
            }
        }
        __syncthreads();  // sdot is refilled by the next group
    }
}

// Kept probes: one warp per query, 32 ranks at a time by ballot (rank 0 and
// every rank whose keep probability exceeds theta), in rank order, then -1.
__global__ void k_prune_compact(const int32_t* __restrict__ probes, int64_t nq, int Pmax,
                                const int32_t* __restrict__ nprobe, int P, const float* __restrict__ prob,
                                float theta, int32_t* __restrict__ probes_out, int32_t* __restrict__ nprobe_out) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nq) return;
    int Pq = nprobe ? nprobe[q] : P;
    Pq = Pq < 1 ? 1 : (Pq > Pmax ? Pmax : Pq);
    int kept = 0;
    for (int r0 = 0; r0 < Pq; r0 += 32) {
        const int r = r0 + lane;
        const bool keep = r < Pq && (r == 0 || prob[q * Pmax + r] > theta);
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        if (keep) probes_out[q * Pmax + kept + __popc(m & ((1u << lane) - 1u))] = probes[q * Pmax + r];
        kept += __popc(m);
    }
    for (int r = kept + lane; r < Pmax; r += 32) probes_out[q * Pmax + r] = -1;
    if (lane == 0 && nprobe_out) nprobe_out[q] = kept;
}

int prune_rows(ksc_index* ix, const float* Q, int64_t nq, const int32_t* probes, int Pmax, const int32_t* nprobe,
               int P, float theta, float* feats, float* prob, int32_t* probes_out, int32_t* nprobe_out,
               cudaStream_t st) {
    KSC_CHECK_STATE(ix->pr_have_stats, "the pruning statistics have not been computed");
    const bool need_model = prob || probes_out || nprobe_out;
    KSC_CHECK_STATE(!need_model || ix->pr_model, "no pruning model");
    KSC_CHECK_ARG(!nprobe_out || probes_out, "nprobe_out needs probes_out");
    if (nq == 0) return KSC_OK;
    if (probes_out && !prob) {  // the probabilities only feed the compaction
        KSC_TRY(ensure(ix->ws_pprob, sizeof(float) * nq * Pmax, st));
        prob = (float*)ix->ws_pprob.p;
    }
    PruneArgs A{Q, nq, ix->d, ix->L, ix->c_mean, probes, Pmax, nprobe, P, ix->pr_stats, ix->pr_vecs,
                need_model ? ix->pr_model : nullptr, theta, feats, prob, probes_out, nprobe_out};
    KSC_CHECK_ARG(Pmax <= PR_ROWS, "pruning needs nprobe <= %d", PR_ROWS);
    const int QB = PR_ROWS / Pmax;
    const int64_t groups = (nq + QB - 1) / QB;
    const unsigned grid = (unsigned)std::min<int64_t>(groups, (int64_t)num_sms() * 2);  // 2 CTAs fit per SM
    if (ix->d <= 128) k_prune_rows<4><<<grid, PR_ROWS, 0, st>>>(A);
    else if (ix->d <= 256) k_prune_rows<8><<<grid, PR_ROWS, 0, st>>>(A);
    else if (ix->d <= 512) k_prune_rows<16><<<grid, PR_ROWS, 0, st>>>(A);
    else k_prune_rows<32><<<grid, PR_ROWS, 0, st>>>(A);
    KSC_LAUNCH_CHECK();
    if (probes_out) {
        k_prune_compact<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(probes, nq, Pmax, nprobe, P, prob, theta,
                                                                   probes_out, nprobe_out);
        KSC_LAUNCH_CHECK();
    }
    return KSC_OK;
}

// ------------------------------------------------------------------ training pieces
// Labels: one warp per query, 32 returned results at a time; a probe rank is
// labelled 1 when any true neighbour among them lies in its list.
__global__ void k_prune_labels(const int64_t* __restrict__ ids, const float* __restrict__ dists, int64_t nq, int k,
                               const float* __restrict__ kth, int ip, const int32_t* __restrict__ assign,
                               const int32_t* __restrict__ probes, int Pmax, int P, float* __restrict__ label) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nq) return;
    const float t = kth[q];
    const float tol = 1e-5f * fabsf(t) + 1e-6f;
    const int32_t* pr = probes + q * Pmax;
    float* lab = label + q * Pmax;
    for (int r = lane; r < Pmax; r += 32) lab[r] = 0.f;
    __syncwarp();
    for (int j0 = 0; j0 < k; j0 += 32) {
        const int j = j0 + lane;
        bool hit = false;
        int a = -1;
        if (j < k) {
            const int64_t id = ids[q * k + j];
            const float dv = dists[q * k + j];
            hit = id >= 0 && (ip ? (dv >= t - tol) : (dv <= t + tol));
            if (hit) a = assign[id];
        }
        for (int r = 0; r < P && r < Pmax; ++r)
            if (__any_sync(0xffffffffu, hit && a == pr[r]) && lane == 0) lab[r] = 1.f;
    }
}

int prune_labels(ksc_index* ix, const int64_t* ids, const float* dists, int64_t nq, int k, const float* kth,
                 const int32_t* probes, int Pmax, int P, float* label, cudaStream_t st) {
    if (nq == 0) return KSC_OK;
    k_prune_labels<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(ids, dists, nq, k, kth, ix->metric == KSC_IP,
                                                             ix->assign, probes, Pmax, P, label);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

// Mean and standard deviation (floored at 1e-6) of feature f = blockIdx.x over
// `rows` rows, FP64, fixed order; written into the model after the weights.
__global__ void __launch_bounds__(256) k_prune_moments(const float* __restrict__ x, int64_t rows,
                                                       float* __restrict__ model) {
    __shared__ double red[PR_WARPS];
    const int f = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) s += x[i * PR_NF + f];
    const double mean = block_sum_d(s, red) / (double)(rows > 0 ? rows : 1);
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
        const double e = x[i * PR_NF + f] - mean;
        v += e * e;
    }
    const double var = block_sum_d(v, red) / (double)(rows > 0 ? rows : 1);
    if (threadIdx.x == 0) {
        model[PR_NP + f] = (float)mean;
        model[PR_NP + PR_NF + f] = (float)fmax(sqrt(var), 1e-6);
    }
}

__global__ void k_prune_standardise(float* __restrict__ x, int64_t rows, const float* __restrict__ model) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * PR_NF) return;
    const int f = (int)(e % PR_NF);
    x[e] = (x[e] - model[PR_NP + f]) / model[PR_NP + PR_NF + f];
}

// Both heads of a row train on its label.
__global__ void k_prune_targets(const float* __restrict__ lab, int64_t rows, float* __restrict__ y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    y[2 * i] = lab[i];
    y[2 * i + 1] = lab[i];
}

int prune_standardise(float* x, int64_t rows, float* model, cudaStream_t st) {
    k_prune_moments<<<PR_NF, 256, 0, st>>>(x, rows, model);
    k_prune_standardise<<<(unsigned)((rows * PR_NF + 255) / 256), 256, 0, st>>>(x, rows, model);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

int prune_targets(const float* lab, int64_t rows, float* y, cudaStream_t st) {
    k_prune_targets<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(lab, rows, y);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

}  // namespace ksc
