// Component filtration (Sec. 4.3; Alg. 1 and Alg. 2 FilterComponents).
//
// For every dimension t of the base vectors: the mean mu_t, the population
// standard deviation sigma_t and the fraction of values that are 0 or within
// one standard deviation of the mean.  Dimensions whose fraction exceeds the
// threshold are dropped from the base vectors and from every query before
// ranking, tables and scan; the exact re-rank keeps the full vectors.
//
// Three passes over the rows (sum, squared deviation, count), each as
// per-chunk partial sums in FP64 (a thread per column, rows of a chunk in
// order, so reads are coalesced across the threads) reduced over the chunks
// in a fixed order: the result does not depend on scheduling.
#include "index.cuh"

namespace ksc {

constexpr int CF_ROWS = 1024;  // rows per chunk
constexpr int CF_T = 256;      // columns per CTA

// mode 0: sum of x; 1: sum of (x - mu)^2; 2: count of x == 0 or |x - mu| <= sigma
__global__ void __launch_bounds__(CF_T) k_col_partial(const float* __restrict__ X, int64_t n, int d, int mode,
                                                      const double* __restrict__ mu, const double* __restrict__ sd,
                                                      double* __restrict__ part) {
    const int t = blockIdx.x * CF_T + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * CF_ROWS;
    if (t >= d) return;
    const int64_t r1 = r0 + CF_ROWS < n ? r0 + CF_ROWS : n;
    const double m = mode > 0 ? mu[t] : 0.0, s = mode > 1 ? sd[t] : 0.0;
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
        const double x = (double)X[r * d + t];
        if (mode == 0) acc += x;
        else if (mode == 1) acc += (x - m) * (x - m);
        else acc += (x == 0.0 || fabs(x - m) <= s) ? 1.0 : 0.0;
    }
    part[(int64_t)blockIdx.y * d + t] = acc;
}

__global__ void k_col_finish(const double* __restrict__ part, int64_t nchunk, int64_t n, int d, int mode,
                             double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d) return;
    double acc = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) acc += part[c * d + t];
    const double nn = n > 0 ? (double)n : 1.0;
    out[t] = mode == 1 ? sqrt(acc / nn) : acc / nn;  // mean, std, fraction
}

// out[r][j] = A[r][dims[j]] (0 where dims[j] < 0), rows of width dw.
__global__ void k_gather_dims(const float* __restrict__ A, int64_t rows, int d, const int32_t* __restrict__ dims,
                              int dw, float* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * dw) return;
    const int64_t r = e / dw;
    const int j = (int)(e - r * dw);
    const int t = dims[j];
    out[e] = t >= 0 ? A[r * d + t] : 0.f;
}

int component_stats(const float* X, int64_t n, int d, double* mu, double* sd, double* frac, cudaStream_t st) {
    const int64_t nchunk = (n + CF_ROWS - 1) / CF_ROWS;
    KSC_CHECK_ARG(nchunk <= 65535, "too many rows for the column statistics (%lld)", (long long)n);
    double* part = nullptr;
    KSC_CUDA(cudaMalloc(&part, sizeof(double) * nchunk * d + 16));
    const dim3 grid((unsigned)((d + CF_T - 1) / CF_T), (unsigned)nchunk);
    double* outs[3] = {mu, sd, frac};
    int rc = KSC_OK;
    for (int mode = 0; mode < 3 && rc == KSC_OK; ++mode) {
        k_col_partial<<<grid, CF_T, 0, st>>>(X, n, d, mode, mu, sd, part);
        k_col_finish<<<(unsigned)((d + 255) / 256), 256, 0, st>>>(part, nchunk, n, d, mode, outs[mode]);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("component statistics: %s", cudaGetErrorString(e));
            rc = KSC_ECUDA;
        }
    }
    cudaStreamSynchronize(st);  // part is freed below
    cudaFree(part);
    return rc;
}

int gather_dims(const float* A, int64_t rows, int d, const int32_t* dims, int dw, float* out, cudaStream_t st) {
    if (rows == 0) return KSC_OK;
    k_gather_dims<<<(unsigned)((rows * dw + 255) / 256), 256, 0, st>>>(A, rows, d, dims, dw, out);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

}  // namespace ksc
