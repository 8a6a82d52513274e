// The predictor network's layout and the device arithmetic shared by its
// kernels (mlp.cu) and the fused ranking + predictor kernel (search.cu):
// parameter views, the feature distance, BF16 rounding and the maps from the
// heads' probabilities to nprobe and R (Eq. 2, or the regression heads').
#pragma once
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

namespace ksc {

constexpr int MLP_F = 64, MLP_H = 64, MLP_O = 2, MLP_FEAT_K = 32;
constexpr int MLP_NPARAM = MLP_H * MLP_F + MLP_H + MLP_H * MLP_H + MLP_H + MLP_O * MLP_H + MLP_O;

struct MlpW {  // views into a packed parameter vector (same packing as the oracle)
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};
// Network F -> H -> H -> 2: parameter count and views.
template <int F, int H>
constexpr int mlp_nparam() {
    return H * F + H + H * H + H + MLP_O * H + MLP_O;
}
template <int F, int H>
__host__ __device__ inline MlpW mlp_views_t(const float* w) {
    MlpW v;
    v.W1 = w;
    v.b1 = v.W1 + H * F;
    v.W2 = v.b1 + H;
    v.b2 = v.W2 + H * H;
    v.W3 = v.b2 + H;
    v.b3 = v.W3 + MLP_O * H;
    return v;
}
__host__ __device__ inline MlpW mlp_views(const float* w) { return mlp_views_t<MLP_F, MLP_H>(w); }

// The distance a ranking score stands for in the features: the score (L2,
// the query's squared norm included) or 1 + s (spherical, s = -<q, c>).
__device__ __forceinline__ float feat_dist(float s, int spherical) { return spherical ? 1.f + s : s; }

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Eq. 2 with the line-broken product read literally:
// P = min(Pmax, Pmin + ceil((Pmax - Pmin) * max(0, p - p0) * (p + p1))).
__host__ __device__ inline int eq2(float p, int pmin, int pmax, float p0, float p1) {
    const float relu = p - p0 > 0.f ? p - p0 : 0.f;
    const float v = ceilf((float)(pmax - pmin) * relu * (p + p1));
    const float r = (float)pmin + v;
    return r > (float)pmax ? pmax : (r < (float)pmin ? pmin : (int)r);
}

// Regression heads: p is the normalised log of the setting,
// u = clamp(p (1 + b) + a, 0, 1), P = clamp(ceil(lo (hi / lo)^u - 1e-3), lo, hi)
// (a value within 1e-3 above an integer counts as that integer).
__device__ inline int regmap(float p, int lo, int hi, float a, float b) {
    const float u = fminf(fmaxf(p * (1.f + b) + a, 0.f), 1.f);
    const float v = (float)lo * powf((float)hi / (float)lo, u);
    const float r = ceilf(v - 1e-3f);
    return r > (float)hi ? hi : (r < (float)lo ? lo : (int)r);
}

}  // namespace ksc
