// Arguments and device helpers shared by the scan kernels: the byte-permute
// scans, thresholds and selections (search.cu) and the tensor-core scan
// (scan_tc.cu).  Work lists are cluster-major: pairs of (query, probe rank)
// grouped by list, items = (list, query group, tile of the list's blocks).
#pragma once

#include "index.cuh"

namespace ksc {

struct ScanArgs {
    int M;
    int Pmax;
    int64_t nq;
    const int32_t* probes;
    const int32_t* nprobe_q;
    int Pfix;
    const int32_t* rerank_q;
    int Rfix, Rmin;
    const uint8_t* lut;
    const int32_t* bias;
    const int64_t* boff;
    const int32_t* list_n;
    const uint8_t* codes;
    const int32_t* ids;
    int L;
};

__device__ __forceinline__ int nprobe_of(const ScanArgs& A, int64_t q) {
    int P = A.nprobe_q ? A.nprobe_q[q] : A.Pfix;
    return P < 1 ? 1 : (P > A.Pmax ? A.Pmax : P);
}

__device__ __forceinline__ int rerank_of(const int32_t* rerank_q, int Rfix, int Rmin, int Rmax, int64_t q) {
    int R = rerank_q ? rerank_q[q] : Rfix;
    return R < Rmin ? Rmin : (R > Rmax ? Rmax : R);
}

__device__ __forceinline__ int64_t list_size(const ScanArgs& A, int p) {
    return (p >= 0 && p < A.L) ? A.list_n[p] : 0;
}

// Place of the first key of probe rank r in query q's unfiltered store: the
// keys of its lower ranks come first.
__device__ __forceinline__ int64_t near_offset(const ScanArgs& A, int64_t q, int r) {
    const int32_t* pr = A.probes + q * A.Pmax;
    int64_t off = 0;
    for (int r2 = 0; r2 < r; ++r2) off += list_size(A, pr[r2]);
    return off;
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(s));
    return r;
}

// Packed FP32 pairs (sm_100 family): each half is the IEEE single-precision
// operation rounded to nearest, the same result as the scalar instruction,
// in one instruction for both.
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

struct ScanOut {
    const uint64_t* thr;
    int32_t* cnt;
    uint64_t* cand;
    int cap;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

struct ScanItem {
    int p, b0, b1;
    int64_t g0, npairs;
};

// Item `it` of a work list, by the whole warp: the last list p with
// item_off[p] <= it is found by a 32-way search (each round one load per lane
// and a ballot; two rounds for 1024 lists), then the item's query group and
// tile.  All 32 lanes call and get the same item.
__device__ __forceinline__ ScanItem locate_item(const ScanArgs& A, const int64_t* __restrict__ pair_off,
                                                const int64_t* __restrict__ item_off, int L, int TB, int QG,
                                                int64_t it, int unit = 1) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = L - 1;  // invariant: item_off[lo] <= it < item_off[hi + 1]
    while (lo < hi) {
        const int step = (hi - lo + 32) / 32;  // ceil((hi - lo + 1) / 32)
        const int pos = min(lo + lane * step, hi);
        const uint32_t m = __ballot_sync(0xffffffffu, item_off[pos] <= it);  // a prefix of lanes; lane 0 holds
        const int last = 31 - __clz(m);
        const int nlo = min(lo + last * step, hi);
        hi = (last < 31 && lo + (last + 1) * step <= hi) ? lo + (last + 1) * step - 1 : hi;
        lo = nlo;
    }
    ScanItem r;
    r.p = lo;
    const int nb = (A.list_n[lo] + 31) >> 5;
    const int nt = (nb + TB - 1) / TB;
    const int64_t local = it - item_off[lo];
    const int64_t grp = local / nt;
    const int tile = (int)(local - grp * nt);
    // the list's nt tiles of near-equal length in whole units (no tile is
    // empty: there are at least nt units)
    const int nu = (nb + unit - 1) / unit;
    r.b0 = (int)((int64_t)tile * nu / nt) * unit;
    r.b1 = min(nb, (int)((int64_t)(tile + 1) * nu / nt) * unit);
    r.g0 = pair_off[lo] + grp * QG;
    r.npairs = pair_off[lo + 1] - r.g0;
    return r;
}

// The tensor-core scan (scan_tc.cu): queries per item for M subspaces (0: not
// supported), and one launch over a work list of items of at most nt queries
// and TB blocks (whole 4-block units).
int tcs_nt(int M);
int launch_scan_tc(const ScanArgs& A, const ScanOut& O, const int64_t* pair_off, const int64_t* item_off,
                   const uint32_t* pairs, int L, int TB, int nt, unsigned long long* next_item, int32_t* status,
                   cudaStream_t st);

}  // namespace ksc
