// The LUT16 scan on the 5th-generation tensor cores (Alg. 3's table lookups
// as a matrix product; opt-in through ksc_search_opts.scan_tc).
#include <algorithm>

#include "scan.cuh"

namespace ksc {

// ------------------------------------------------------------------ a3: LUT16 scan on the tensor cores
// The lookup sums of one list for a group of queries as one matrix product.
// A (row = vector, K = 16 M): entry 16 j + c is 1 when the vector's code in
// subspace j is c, else 0.  B (row = query): entry 16 j + e is 1024 + T_j[e],
// T the query's u8 table of the list.  Row v of A B^T for query n is then
// 1024 M + sum_j T_j[c_j(v)]: an integer below 2^17, exact in the FP32
// accumulator whatever the order of the additions, so the keys equal those of
// the byte-permute scan bit for bit.  Both operands are FP16 (1.0 and the
// integers 1024 .. 1279 are exact), M 128 vectors x N queries x K 16 per
// tcgen05.mma.
//
// A is never in memory: the threads expand each 128-vector tile's codes into
// tensor memory with tcgen05.st (lane = vector, two K entries per 32-bit
// column), eight subspaces (64 columns) per chunk, and the MMAs read it there.
// B, the item's tables, is staged once per item into shared memory (K-major,
// 128-byte swizzle, boxes of 64 K entries) and read by every tile of the item.
// Roles: two warpgroups expand alternate chunks of every tile, each into its
// own ring of TMEM slots, and split the tile's epilogue (reading the
// accumulator: lane = vector, column = query; testing / writing the keys) by
// 16-column groups; one more warp issues the MMAs.  mbarriers: a chunk
// written (128 arrivals), a chunk read (tcgen05.commit), a tile's product
// complete (tcgen05.commit), an accumulator read by both warpgroups (256
// arrivals).  Every wait is bounded.
constexpr int TCS_NT = 64;        // queries per item (B rows, MMA N <= 64)
constexpr int TCS_SLOTS = 3;      // TMEM chunk slots per warpgroup
constexpr int TCS_THREADS = 288;  // two warpgroups + the MMA warp
constexpr int TCS_TMEM_COLS = 512;
constexpr int TCS_D_COL = 0;      // two accumulators, tiles alternating: accumulator b at column b * TCS_NT
constexpr int TCS_A_COL = 2 * TCS_NT;  // chunk slots: (g * TCS_SLOTS + s) * 64 after the accumulators
constexpr uint32_t TCS_WAIT = 1u << 22;
constexpr int TCS_KCAP = 64;      // passing keys buffered in shared memory per query column and item
static_assert(TCS_A_COL + 2 * TCS_SLOTS * 64 <= TCS_TMEM_COLS, "tensor memory columns");

struct TcsQuery {
    int64_t q, noff;
    uint32_t e, thI;
    int32_t bias, lim;
};

// Bounded wait on an mbarrier phase: a few quick polls, then polls spaced by
// a short sleep, so that a waiting warp does not take issue slots from the
// warps of its scheduler that have work (at most TCS_WAIT polls).
__device__ __forceinline__ bool tcs_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < TCS_WAIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i >= 4) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tcs_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tcs_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// K-major operand in shared memory, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t tcs_sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// kind::f16 instruction descriptor: FP16 A and B, FP32 D, both K-major, M 128 x N
__device__ __forceinline__ uint32_t tcs_idesc(int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// D[tmem d] (+)= A[tmem a] B[smem desc b]^T
__device__ __forceinline__ void tcs_mma(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(
            d),
        "r"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tcs_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tcs_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared memory of k_scan_tc: B (Mc boxes of nt rows x 128 bytes), then per
// generating warp the transposed codes of its block (4 words x 4 Mc
// subspaces: word w of subspace j holds the codes of vectors 8 w .. 8 w + 7),
// then the filtered scan's key buffers (TCS_KCAP keys per query column).
__host__ __device__ inline size_t tcs_smem_bytes(int M, int nt) {
    const int Mc = (M + 3) / 4, Mw = (M + 7) / 8 * 8;
    return 1024 + (size_t)Mc * nt * 128 + (size_t)8 * 4 * Mw * 4 + (size_t)nt * TCS_KCAP * 8;
}

// Items = (list p, group of at most nt queries probing p, tile [b0, b1) of
// p's blocks, whole 4-block units), taken in turn from a global counter.
// Both warpgroups work on the same 128-vector tile: warpgroup g expands the
// chunks c = g, g + 2, ... (warp w4 the vectors of block 4 mt + w4, lanes
// 32 w4 .. 32 w4 + 31 of tensor memory) and reads the query columns of the
// 16-column groups g, g + 2, ... of the accumulator.  Two accumulators
// alternate between tiles: a tile's epilogue runs after the next tile's
// chunks are written, so the MMAs of the next tile overlap it; an mbarrier
// tells the MMA warp when both warpgroups are done with an accumulator.
template <bool DIRECT>
__global__ void __launch_bounds__(TCS_THREADS, 1)
    k_scan_tc(ScanArgs A, ScanOut O, const int64_t* __restrict__ pair_off, const int64_t* __restrict__ item_off,
              const uint32_t* __restrict__ pairs, int L, int TB, int nt, unsigned long long* __restrict__ next_item,
              int32_t* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t tcs_raw[];
    __shared__ __align__(8) uint64_t bar_full[2][TCS_SLOTS], bar_free[2][TCS_SLOTS], bar_dfull[2], bar_dfree[2],
        bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ ScanItem s_x;
    __shared__ long long s_it;
    __shared__ int s_fail;
    __shared__ TcsQuery s_q[TCS_NT];
    __shared__ int s_kc[TCS_NT];  // keys reserved in each query column's shared buffer (this item)
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tcs_raw) + 1023) & ~uintptr_t(1023));
    // Mc boxes of 4 subspaces (B), Mc8 chunks of 8 subspaces (A), transposed
    // code rows of Mw words
    const int M = A.M, Mc = (M + 3) / 4, Mc8 = (M + 7) / 8, Mw = Mc8 * 8;
    const uint32_t box = (uint32_t)nt * 128;
    const uint32_t sB = smem_addr(smem);
    uint32_t* trans = reinterpret_cast<uint32_t*>(smem + (size_t)Mc * box);
    uint64_t* kbuf = reinterpret_cast<uint64_t*>(trans + (size_t)8 * 4 * Mw);  // [nt][TCS_KCAP]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int g = 0; g < 2; ++g) {
            for (int s = 0; s < TCS_SLOTS; ++s) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_addr(&bar_full[g][s])) : "memory");
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_free[g][s])) : "memory");
            }
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_dfull[g])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;" ::"r"(smem_addr(&bar_dfree[g])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_drain)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (tid < TCS_NT) s_kc[tid] = 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(TCS_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int64_t total = item_off[L];
    const int bias1024 = 1024 * M;
    const int g = warp >> 2, w4 = warp & 3;
    // pipeline counters, the same sequence on every side: chunks written by
    // warpgroup g (kc; MMA side kcm0 / kcm1) and tiles (tcount)
    uint32_t kc = 0, kcm0 = 0, kcm1 = 0, tcount = 0;
    while (true) {
        if (tid == 0) s_it = (long long)atomicAdd(next_item, 1ull);
        __syncthreads();
        const int64_t it = s_it;
        if (it >= total || s_fail) break;
        if (warp == 0) {
            const ScanItem x = locate_item(A, pair_off, item_off, L, TB, nt, it, 4);
            if (lane == 0) s_x = x;
        }
        __syncthreads();
        const ScanItem x = s_x;
        const int nqi = (int)(x.npairs < nt ? x.npairs : nt);
        const int N = (nqi + 15) & ~15;
        const int listn = A.list_n[x.p];
        const int64_t gb = A.boff[x.p];
        if (tid < nqi) {
            TcsQuery qi;
            qi.e = pairs[x.g0 + tid];
            qi.q = qi.e / A.Pmax;
            qi.noff = DIRECT ? near_offset(A, qi.q, (int)(qi.e - qi.q * A.Pmax)) : 0;
            qi.bias = A.bias[qi.e];
            const uint64_t th = O.thr ? O.thr[qi.q] : KEY_NONE;
            qi.thI = (uint32_t)th;
            const int64_t l = (int64_t)(th >> 32) - 2147483648ll - qi.bias;
            qi.lim = (int32_t)(l < -1 ? -1 : (l > (1 << 24) ? (1 << 24) : l));
            s_q[tid] = qi;
        }
        __syncthreads();
        // B: row n, K entry 16 j + e = FP16 (1024 + T_j[e]) (bits 0x6400 | T);
        // rows nqi .. N-1 and subspaces M .. 4 Mc - 1 are zero.  Four table
        // rows per thread in flight.
        {
            const int tot = N * 4 * Mc;
            for (int i0 = tid; i0 < tot; i0 += 4 * TCS_THREADS) {
                uint4 t[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int idx = i0 + u * TCS_THREADS;
                    const int n = idx / (4 * Mc), j = idx - n * (4 * Mc);
                    t[u] = (idx < tot && n < nqi && j < M)
                               ? __ldg(reinterpret_cast<const uint4*>(A.lut + (int64_t)s_q[n].e * M * PQ_K) + j)
                               : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int idx = i0 + u * TCS_THREADS;
                    if (idx >= tot) break;
                    const int n = idx / (4 * Mc), j = idx - n * (4 * Mc);
                    const uint32_t hb = (n < nqi && j < M) ? 0x64646464u : 0u;
                    const uint4 h0 = make_uint4(prmt(t[u].x, hb, 0x4140u), prmt(t[u].x, hb, 0x4342u),
                                                prmt(t[u].y, hb, 0x4140u), prmt(t[u].y, hb, 0x4342u));
                    const uint4 h1 = make_uint4(prmt(t[u].z, hb, 0x4140u), prmt(t[u].z, hb, 0x4342u),
                                                prmt(t[u].w, hb, 0x4140u), prmt(t[u].w, hb, 0x4342u));
                    const int ch = (j & 3) * 2, sw = n & 7;
                    uint8_t* row = smem + (size_t)(j >> 2) * box + (n >> 3) * 1024 + sw * 128;
                    *reinterpret_cast<uint4*>(row + ((ch ^ sw) << 4)) = h0;
                    *reinterpret_cast<uint4*>(row + (((ch + 1) ^ sw) << 4)) = h1;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        const int nmt = (x.b1 - x.b0 + 3) / 4;
        if (warp == 8) {
            if (lane == 0 && !s_fail) {
                const uint32_t idesc = tcs_idesc(N);
                bool ok = true;
                for (int mt = 0; mt < nmt && ok; ++mt) {
                    const uint32_t b = tcount & 1u;
                    // both warpgroups have read this accumulator's previous tile
                    if (tcount >= 2) ok = tcs_wait(smem_addr(&bar_dfree[b]), ((tcount >> 1) - 1) & 1u);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dcol = tmem + TCS_D_COL + b * TCS_NT;
                    for (int c = 0; c < Mc8 && ok; ++c) {
                        const int gg = c & 1;
                        const uint32_t kk = gg ? kcm1 : kcm0;
                        const uint32_t s = kk % TCS_SLOTS, u = kk / TCS_SLOTS;
                        ok = tcs_wait(smem_addr(&bar_full[gg][s]), u & 1u);
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t acol = tmem + TCS_A_COL + (gg * TCS_SLOTS + s) * 64;
#pragma unroll
                        for (int uu = 0; uu < 8; ++uu)
                            if (2 * c + (uu >> 2) < Mc)  // the last chunk of an odd box count has one box
                                tcs_mma(dcol, acol + uu * 8, tcs_sdesc(sB + (2 * c + (uu >> 2)) * box + (uu & 3) * 32),
                                        idesc, (c | uu) != 0);
                        tcs_commit(smem_addr(&bar_free[gg][s]));
                        if (gg) kcm1 = kk + 1;
                        else kcm0 = kk + 1;
                    }
                    if (ok) tcs_commit(smem_addr(&bar_dfull[b]));
                    ++tcount;
                }
                if (!ok) {
                    atomicOr(status, 8);
                    s_fail = 1;
                }
            }
            __syncwarp();
        } else {
            uint32_t* tr = trans + (size_t)warp * 4 * Mw;
            const uint32_t* mine = tr + (lane >> 3) * Mw;
            const int sh = 4 * (lane & 7);
            const uint32_t lane_addr = (uint32_t)(32 * w4) << 16;
            bool ok = true;
            // the codes of this warp's block of tile mt, four rows per lane
            uint4 rows[4];
            auto load_rows = [&](int mt) {
                const int blk = x.b0 + 4 * mt + w4;
                const bool vb = mt < nmt && blk < x.b1;
                const uint4* src = reinterpret_cast<const uint4*>(A.codes + (gb + blk) * (int64_t)M * 16);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = lane + 32 * u;
                    rows[u] = (vb && j < M) ? __ldg(src + j) : make_uint4(0, 0, 0, 0);
                }
            };
            // expand subspaces 4 q .. 4 q + 3 of the current codes into r
            auto expand = [&](int q4, uint32_t(&r)[32]) {
                const uint4 wv = *reinterpret_cast<const uint4*>(mine + 4 * q4);
                const uint32_t wd[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                for (int uu = 0; uu < 4; ++uu) {
                    const uint32_t code = (wd[uu] >> sh) & 15u;
                    const uint32_t h = code >> 1;
                    const uint32_t val = (4 * q4 + uu < M) ? (0x3C00u << ((code & 1u) << 4)) : 0u;
#pragma unroll
                    for (int i = 0; i < 8; ++i) r[8 * uu + i] = h == (uint32_t)i ? val : 0u;
                }
            };
            // epilogue of tile t (global tile number T): this warpgroup's
            // 16-column groups of accumulator T & 1
            auto epilogue = [&](int t, uint32_t T, uint32_t id) {
                const uint32_t b = T & 1u;
                if (ok) ok = __all_sync(0xffffffffu, tcs_wait(smem_addr(&bar_dfull[b]), (T >> 1) & 1u));
                if (ok) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int blk = x.b0 + 4 * t + w4;
                    const int vidx = blk * 32 + lane;
                    const bool valid = blk < x.b1 && vidx < listn;
                    for (int n0 = 16 * g; n0 < nqi; n0 += 32) {
                        uint32_t f[16];
                        tcs_ld16(tmem + lane_addr + TCS_D_COL + b * TCS_NT + n0, f);
                        if (DIRECT) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const int n = n0 + i;
                                if (n >= nqi) break;
                                const TcsQuery& qi = s_q[n];
                                const int32_t sum = __float2int_rz(__uint_as_float(f[i])) - bias1024;
                                const uint64_t key =
                                    ((uint64_t)((uint32_t)(qi.bias + sum) ^ 0x80000000u) << 32) | (uint64_t)id;
                                const int64_t pos = qi.noff + vidx;
                                if (valid && pos < O.cap) O.cand[qi.q * O.cap + pos] = key;
                            }
                        } else {
                            // this lane's vector against the 16 columns, without
                            // branches (independent tests, so their latencies
                            // overlap): pass bits, then per column a ballot,
                            // one shared reservation per column by lane i for
                            // column n0 + i (all 16 at once), and the stores
                            // into the column's shared buffer -- or, for what
                            // does not fit there, into the global store
                            uint32_t pm = 0;
                            int32_t sums[16];
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const int n = n0 + i;  // < TCS_NT: n0 <= TCS_NT - 16
                                sums[i] = __float2int_rz(__uint_as_float(f[i])) - bias1024;
                                const int32_t lim = s_q[n].lim;
                                const uint32_t th = s_q[n].thI;
                                const bool pass = n < nqi && valid && (sums[i] < lim || (sums[i] == lim && id <= th));
                                pm |= (uint32_t)pass << i;
                            }
                            uint32_t bal[16];
                            int cnt = 0;
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                bal[i] = __ballot_sync(0xffffffffu, (pm >> i) & 1u);
                                cnt = lane == i ? __popc(bal[i]) : cnt;
                            }
                            int sb = 0, gb = 0;
                            if (cnt > 0) {
                                sb = atomicAdd(&s_kc[n0 + lane], cnt);
                                const int fit = max(0, min(cnt, TCS_KCAP - sb));
                                if (cnt > fit) gb = atomicAdd(&O.cnt[s_q[n0 + lane].q], cnt - fit);
                            }
                            const uint32_t below = (1u << lane) - 1u;
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                if (bal[i] == 0u) continue;  // the same on every lane
                                const int sbi = __shfl_sync(0xffffffffu, sb, i);
                                const int gbi = __shfl_sync(0xffffffffu, gb, i);
                                if ((pm >> i) & 1u) {
                                    const int n = n0 + i;
                                    const uint64_t key =
                                        ((uint64_t)((uint32_t)(s_q[n].bias + sums[i]) ^ 0x80000000u) << 32) |
                                        (uint64_t)id;
                                    const int p = sbi + __popc(bal[i] & below);
                                    if (p < TCS_KCAP) {
                                        kbuf[n * TCS_KCAP + p] = key;
                                    } else {
                                        const int at = gbi + (p - max(sbi, TCS_KCAP));
                                        if (at < O.cap) O.cand[s_q[n].q * O.cap + at] = key;
                                    }
                                }
                            }
                        }
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                }
                tcs_arrive(smem_addr(&bar_dfree[b]));
            };
            load_rows(0);
            uint32_t id_prev = 0;
            for (int mt = 0; mt < nmt; ++mt) {
                const int blk = x.b0 + 4 * mt + w4;
                const uint32_t id_cur = (blk < x.b1 && blk * 32 + lane < listn) ? (uint32_t)A.ids[(gb + blk) * 32 + lane] : 0u;
                // transpose this tile's codes: row j (vector v's code in nibble v)
                // -> word v / 8 of subspace j; then fetch the next tile's
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = lane + 32 * u;
                    if (j < M) {
                        tr[0 * Mw + j] = rows[u].x;
                        tr[1 * Mw + j] = rows[u].y;
                        tr[2 * Mw + j] = rows[u].z;
                        tr[3 * Mw + j] = rows[u].w;
                    }
                }
                __syncwarp();
                load_rows(mt + 1);
                // this warpgroup's chunks (8 subspaces, 64 columns): the second
                // half is expanded while the store of the first is in flight
                for (int c = g; c < Mc8 && ok; c += 2) {
                    const uint32_t s = kc % TCS_SLOTS, u = kc / TCS_SLOTS;
                    if (u > 0) {
                        ok = __all_sync(0xffffffffu, tcs_wait(smem_addr(&bar_free[g][s]), (u - 1) & 1u));
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    }
                    const uint32_t col = tmem + lane_addr + TCS_A_COL + (g * TCS_SLOTS + s) * 64;
                    uint32_t ra[32], rb[32];
                    expand(2 * c, ra);
                    tcs_st32(col, ra);
                    expand(2 * c + 1, rb);
                    tcs_st32(col + 32, rb);
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    tcs_arrive(smem_addr(&bar_full[g][s]));
                    ++kc;
                }
                __syncwarp();  // the transposed codes are read before the next tile overwrites them
                if (mt > 0) epilogue(mt - 1, tcount - 1, id_prev);
                id_prev = id_cur;
                ++tcount;
            }
            if (nmt > 0) epilogue(nmt - 1, tcount - 1, id_prev);
            if (!ok && lane == 0) {
                atomicOr(status, 8);
                s_fail = 1;
            }
        }
        __syncthreads();  // the item is done: B, the query table and the counters are free
        if (!DIRECT) {
            // the shared key buffers to the store: one reservation per query
            // column, the copy coalesced by a warp per column
            for (int n = warp; n < nqi; n += TCS_THREADS / 32) {
                const int c = min(s_kc[n], TCS_KCAP);
                int base = 0;
                if (lane == 0 && c > 0) base = atomicAdd(&O.cnt[s_q[n].q], c);
                base = __shfl_sync(0xffffffffu, base, 0);
                for (int i = lane; i < c; i += 32)
                    if (base + i < O.cap) O.cand[s_q[n].q * O.cap + base + i] = kbuf[n * TCS_KCAP + i];
            }
            __syncthreads();
            if (tid < TCS_NT) s_kc[tid] = 0;
        }
    }
    // every MMA issued by this CTA has completed before the tensor memory is freed
    if (tid == 8 * 32) {
        tcs_commit(smem_addr(&bar_drain));
        if (!tcs_wait(smem_addr(&bar_drain), 0)) atomicOr(status, 8);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCS_TMEM_COLS));
}

// Queries per item of the tensor-core scan for M subspaces: the item's tables
// (M x 16 FP16 entries per query) and the transposed codes fit in 200 KB of
// shared memory; 0: not supported (each lane stages at most 4 x 32 code rows
// of a block, so M <= 128).
int tcs_nt(int M) {
    if (M < 1 || M > 128) return 0;
    for (int nt = TCS_NT; nt >= 16; nt -= 16)
        if (tcs_smem_bytes(M, nt) <= 200 * 1024) return nt;
    return 0;
}

// One CTA per SM (the kernel holds all 512 tensor-memory columns; at least
// 120 KB of shared memory keeps a second CTA off the SM).
int launch_scan_tc(const ScanArgs& A, const ScanOut& O, const int64_t* pair_off, const int64_t* item_off,
                   const uint32_t* pairs, int L, int TB, int nt, unsigned long long* next_item, int32_t* status,
                   cudaStream_t st) {
    const size_t smem = std::max<size_t>(tcs_smem_bytes(A.M, nt), 120 * 1024);
    auto kern = O.thr ? k_scan_tc<false> : k_scan_tc<true>;
    KSC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<num_sms(), TCS_THREADS, smem, st>>>(A, O, pair_off, item_off, pairs, L, TB, nt, next_item, status);
    KSC_LAUNCH_CHECK();
    return KSC_OK;
}

}  // namespace ksc
