// Streaming single-pass form (daq_params.grid = -5): every sample is read from
// HBM once; the compaction re-reads each tile's marked columns from L2 shortly
// after the count has brought them there.
//
// One persistent CTA per SM; warps have fixed roles and hand tiles to each
// other through mbarriers over a ring of str_meta tile records in shared
// memory:
//
//   producer     takes a ticket (tiles run in ticket order), decodes the tile
//                and bulk-copies its crystal rows plus halo into one of two
//                count slots (2-D tensor boxes);
//   sum warps    crystal sums (Table 2 row 6) minus the summed pedestals
//                (row 1), threshold bits (row 2) and 8-sample block sums, from
//                the count slot;
//   marks warps  pre/post windows and merge (rows 3-4), the tile aggregate
//                (published for the look-back), Q partial bins (rows 7-8);
//                two warps take alternate tiles;
//   look-back    decoupled look-back over earlier tiles' published states
//                (four warps, tiles in turn): the tile's exclusive prefix (pool
//                row, island index, entering run);
//   loader       once a tile's prefix is known, bulk-copies each 64-sample step
//                of the tile that holds a marked sample (still in L2) into a
//                ring of small step slots;
//   writers      stage the marked samples' rows of each step at their global
//                byte phase (each writer warp owns a fixed set of step slots);
//   store        one bulk copy of the tile's rows plus unaligned ends, and the
//                tile's island records (row 5).
//
// Nothing waits for a tile that was not ticketed earlier, and a ticket is only
// taken when a record and a count slot are free, so every ticketed tile is
// counted and published without waiting on later tiles: the look-backs always
// end.  Every wait is bounded (kWaitLimitNs); a CTA that gives up flags
// DAQ_DEV_TIMEOUT, which makes the other CTAs stop too.
#pragma once

#include "daq_steps.cuh"
#include "daq_twopass.cuh"

namespace daq {

constexpr int kStrProducer = 0;
constexpr int kStrSum0 = 1;
constexpr int kStrNSum = 8;
constexpr int kStrMarks = kStrSum0 + kStrNSum;
constexpr int kStrNMarks = 2;
constexpr int kStrLook = kStrMarks + kStrNMarks;
constexpr int kStrNLook = 4;
constexpr int kStrLoader = kStrLook + kStrNLook;
constexpr int kStrWriter0 = kStrLoader + 1;
constexpr int kStrNWriter = 8;
constexpr int kStrStore = kStrWriter0 + kStrNWriter;
constexpr int kStrWarps = kStrStore + 1;
constexpr int kStrThreads = 32 * kStrWarps;
constexpr int kStrMaxMeta = 8;    // tile records per CTA (a multiple of 4: four look-back warps take turns)
constexpr int kStrNCSlot = 2;     // count slots (extended tile)
constexpr int kStrNQ = 8;         // compaction step slots (64 samples x n_xtal rows)
constexpr int kStrStep = 64;      // samples per compaction step
constexpr int kStrMaxStages = 2;  // row stages (1 or 2, from the shared-memory budget)
static_assert(kStrNQ % kStrNWriter == 0, "every step slot has one owning writer warp");

template <int TW> struct StreamMeta {
    TileInfo T;
    Agg agg, excl;
    uint8_t abyte[128];  // threshold bits of the extended tile
    int32_t blocksum[TW / 8];
    uint32_t wm[TW / 32], ws[TW / 32], we[TW / 32];
    int32_t wmb[TW / 32], wsb[TW / 32], wls[TW / 32];
};

// mbarrier indices
struct StreamBars {
    int nm, ns;
    __host__ __device__ int bits(int m) const { return m; }
    __host__ __device__ int agg(int m) const { return nm + m; }
    __host__ __device__ int excl(int m) const { return 2 * nm + m; }
    __host__ __device__ int meta_free(int m) const { return 3 * nm + m; }
    __host__ __device__ int cfull(int s) const { return 4 * nm + s; }
    __host__ __device__ int cempty(int s) const { return 4 * nm + kStrNCSlot + s; }
    __host__ __device__ int qfull(int q) const { return 4 * nm + 2 * kStrNCSlot + q; }
    __host__ __device__ int qempty(int q) const { return 4 * nm + 2 * kStrNCSlot + kStrNQ + q; }
    __host__ __device__ int stage_full(int o) const { return 4 * nm + 2 * kStrNCSlot + 2 * kStrNQ + o; }
    __host__ __device__ int stage_free(int o) const { return 4 * nm + 2 * kStrNCSlot + 2 * kStrNQ + ns + o; }
    __host__ __device__ int count() const { return 4 * nm + 2 * kStrNCSlot + 2 * kStrNQ + 2 * ns; }
};

template <int TW> __host__ __device__ constexpr size_t stream_meta_bytes()
{
    return (sizeof(StreamMeta<TW>) + 15) & ~size_t(15);
}

__host__ __device__ inline size_t stream_stage_bytes(int tw, int X) { return ((size_t)tw * 2 * X + 32 + 15) & ~size_t(15); }
__host__ __device__ inline size_t stream_qslot_bytes(int X) { return ((size_t)X * 2 * kStrStep + 127) & ~size_t(127); }

// Shared-memory layout: count slots, step slots, stages, tile records, sample
// sums (decimation factors that are not multiples of 8), barriers, fill plan,
// end marker.
template <int TW> struct StreamSmem {
    size_t cslot0, qslot0, stage0, meta0, sarr0, bars, fts, lens, end, total;
    __host__ __device__ StreamSmem(int X, int slot_bytes, int need_sarr, int nm, int ns)
    {
        cslot0 = 0;
        qslot0 = cslot0 + (size_t)kStrNCSlot * slot_bytes;
        stage0 = qslot0 + (size_t)kStrNQ * stream_qslot_bytes(X);
        meta0 = stage0 + (size_t)ns * stream_stage_bytes(TW, X);
        sarr0 = meta0 + (size_t)nm * stream_meta_bytes<TW>();
        bars = (sarr0 + (need_sarr ? (size_t)nm * TW * 4 : 0) + 15) & ~size_t(15);
        fts = bars + (size_t)StreamBars{nm, ns}.count() * 8;
        lens = fts + 8 * (size_t)(kPlanSmem + 1);
        end = (lens + 4 * (size_t)kPlanSmem + 15) & ~size_t(15);
        total = (end + 16 + 127) & ~size_t(127);
    }
};

// Bounded mbarrier wait (one thread or a whole warp).  Returns 1 when the phase
// completed, 0 when the stream ended before iteration i (*s_end < i), -1 on
// timeout or when another CTA flagged one.
__device__ __forceinline__ int stream_wait(const KArgs &a, uint64_t *bar, uint32_t parity, long long i,
                                           const volatile long long *s_end)
{
    if (mbar_try_wait(bar, parity)) return 1;
    const uint64_t t0 = global_ns();
    for (uint32_t k = 0;; ++k) {
        if (mbar_try_wait_sleep(bar, parity, 2000u)) return 1;
        if (s_end && *s_end < i) return 0;
        if ((k & 15u) == 15u) {
            if (global_ns() - t0 > kWaitLimitNs) {
                set_status_bit(a, DAQ_DEV_TIMEOUT);
                return -1;
            }
            if (aborted(a)) return -1;
        }
    }
}

// Warp-uniform form of stream_wait (lane 0's outcome).
__device__ __forceinline__ int stream_wait_warp(const KArgs &a, uint64_t *bar, uint32_t parity, long long i,
                                                const volatile long long *s_end)
{
    int r = stream_wait(a, bar, parity, i, s_end);
    return __shfl_sync(kFull, r, 0);
}

// 64-sample compaction steps of a tile that hold a marked sample: bit j set
// when marks words 2j or 2j + 1 are non-zero (one warp; the result is
// warp-uniform).
template <int TW> __device__ __forceinline__ uint32_t marked_steps(const uint32_t *wm, int lane)
{
    constexpr int NWT = TW / 32;
    const uint32_t b = __ballot_sync(kFull, lane < NWT && wm[lane < NWT ? lane : 0] != 0u);
    uint32_t steps = 0;
#pragma unroll
    for (int j = 0; j < (NWT + 1) / 2; ++j) steps |= ((b >> (2 * j)) & 3u) ? (1u << j) : 0u;
    return steps;
}

// Stage the rows of the marked samples of step j (one warp) from its step slot
// (n_xtal rows of 64 samples, pitch 128 bytes): lane L owns tile columns
// c = 64 j + 2L, c + 1; a marked sample's row goes to byte phase + r * 2X of the
// stage, r = its rank among the tile's marked samples.
__device__ __forceinline__ void stage_step(const KArgs &a, uint32_t qslot_s, int j, int nt, const uint32_t *wm,
                                           const int32_t *wmb, unsigned char *stage, int phase, int lane)
{
    const int X = a.n_xtal;
    const int c = kStrStep * j + 2 * lane;
    const int w = c >> 5, bit = c & 31;
    const uint32_t mw = c < nt ? wm[w] : 0u;
    const uint32_t m0 = (mw >> bit) & 1u, m1 = c + 1 < nt ? (mw >> (bit + 1)) & 1u : 0u;
    if (!(m0 | m1)) return;
    const int r0 = wmb[w] + __popc(mw & ((1u << bit) - 1u));
    const int r1 = r0 + (int)m0;
    const uint32_t base = qslot_s + 4u * (uint32_t)lane;
    unsigned char *row0 = stage + phase + (size_t)r0 * 2 * X, *row1 = stage + phase + (size_t)r1 * 2 * X;
    if (!(X & 1)) {
#pragma unroll 3
        for (int x = 0; x < X; x += 2) {
            const uint32_t w0 = lds_u32(base + (uint32_t)(x * 2 * kStrStep));
            const uint32_t w1 = lds_u32(base + (uint32_t)((x + 1) * 2 * kStrStep));
            if (m0) *reinterpret_cast<uint32_t *>(row0 + 2 * x) = __byte_perm(w0, w1, 0x5410);
            if (m1) *reinterpret_cast<uint32_t *>(row1 + 2 * x) = __byte_perm(w0, w1, 0x7632);
        }
    } else {
        for (int x = 0; x < X; ++x) {
            const uint32_t w0 = lds_u32(base + (uint32_t)(x * 2 * kStrStep));
            if (m0) *reinterpret_cast<uint16_t *>(row0 + 2 * x) = (uint16_t)(w0 & 0xffffu);
            if (m1) *reinterpret_cast<uint16_t *>(row1 + 2 * x) = (uint16_t)(w0 >> 16);
        }
    }
}

template <int TW>
__global__ void __launch_bounds__(kStrThreads, 1) daq_stream_kernel(const __grid_constant__ KArgs a)
{
    constexpr int NBT = TW / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int X = a.n_xtal;
    const int NM = a.str_meta, NS = a.str_stages;
    const StreamBars BI{NM, NS};
    const StreamSmem<TW> L(X, a.slot_bytes, a.need_sarr, NM, NS);
    const size_t stage_bytes = stream_stage_bytes(TW, X), qslot_bytes = stream_qslot_bytes(X);
    constexpr size_t meta_bytes = stream_meta_bytes<TW>();
    unsigned char *cslot0 = smem + L.cslot0;
    unsigned char *qslot0 = smem + L.qslot0;
    unsigned char *stage0 = smem + L.stage0;
    unsigned char *meta0 = smem + L.meta0;
    int32_t *sarr0 = reinterpret_cast<int32_t *>(smem + L.sarr0);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    long long *fts_s = reinterpret_cast<long long *>(smem + L.fts);
    int32_t *lens_s = reinterpret_cast<int32_t *>(smem + L.lens);
    volatile long long *s_end = reinterpret_cast<volatile long long *>(smem + L.end);
    auto meta = [&](int m) { return reinterpret_cast<StreamMeta<TW> *>(meta0 + (size_t)m * meta_bytes); };
    auto sarr = [&](int m) { return sarr0 + (a.need_sarr ? m * TW : 0); };
    auto words = [&](int m) {
        StreamMeta<TW> *M = meta(m);
        return TileWords{M->wm, M->ws, M->we, M->wmb, M->wsb, M->wls};
    };
    auto bar = [&](int idx) { return bars + idx; };
    auto par = [](long long i, int n) { return (uint32_t)((i / n) & 1); };           // phase of use i of a ring of n
    auto par_prev = [](long long i, int n) { return (uint32_t)((i / n - 1) & 1); };  // phase of use i - n

    if (tid == 0) *s_end = 0x7fffffffffffffffll;
    const PlanView plan = cache_plan(a, fts_s, lens_s, tid, kStrThreads);
    for (int m = 0; m < NM; ++m)
        for (int i = tid; i < 32; i += kStrThreads) reinterpret_cast<uint32_t *>(meta(m)->abyte)[i] = 0u;
    if (tid == 0) {
        for (int m = 0; m < NM; ++m) {
            mbar_init(bar(BI.bits(m)), kStrNSum);
            mbar_init(bar(BI.agg(m)), 1);
            mbar_init(bar(BI.excl(m)), 1);
            mbar_init(bar(BI.meta_free(m)), 1);
        }
        for (int s = 0; s < kStrNCSlot; ++s) {
            mbar_init(bar(BI.cfull(s)), 1);
            mbar_init(bar(BI.cempty(s)), kStrNSum);
        }
        for (int q = 0; q < kStrNQ; ++q) {
            mbar_init(bar(BI.qfull(q)), 1);
            mbar_init(bar(BI.qempty(q)), 1);
        }
        for (int o = 0; o < NS; ++o) {
            mbar_init(bar(BI.stage_full(o)), kStrNWriter);
            mbar_init(bar(BI.stage_free(o)), 1);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const long long total = plan.fts[a.n_fills];
    const bool skip_isl = (a.flags & DAQ_SKIP_ISLANDS) != 0;
    const bool skip_q = (a.flags & DAQ_SKIP_Q) != 0;

    if (warp == kStrProducer) {
        // ------------------------------------------------------------ tickets, decode, count-slot loads
        if (lane == 0) {
            for (long long i = 0;; ++i) {
                const int m = (int)(i % NM), s = (int)(i % kStrNCSlot);
                if (i >= NM && stream_wait(a, bar(BI.meta_free(m)), par_prev(i, NM), i, nullptr) != 1) break;
                if (i >= kStrNCSlot && stream_wait(a, bar(BI.cempty(s)), par_prev(i, kStrNCSlot), i, nullptr) != 1)
                    break;
                StreamMeta<TW> *M = meta(m);
                const long long tk = (long long)atomicAdd(a.ticket, 1u);
                if (!decode_tile<TW>(a, tk, M->T, plan.fts, plan.lens)) {
                    M->T.tile = -1;
                    *s_end = i;
                    mbar_arrive(bar(BI.cfull(s)));
                    break;
                }
                trace_stamp(a, tk, 0);
                trace_value(a, tk, 10, sm_id());
                trace_value(a, tk, 11, TW);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar(BI.cfull(s)), tile_load_bytes(a));
                issue_tile_load(a, M->T, cslot0 + (size_t)s * a.slot_bytes, bar(BI.cfull(s)));
                trace_stamp(a, tk, 1);
            }
            // the sum warps wait for every load issued, so none is in flight at exit
        }
    } else if (warp >= kStrSum0 && warp < kStrSum0 + kStrNSum) {
        // ------------------------------------------------------------ crystal sums, threshold bits
        const int sw = warp - kStrSum0;
        const int n_steps = (a.ew + 63) / 64;
        for (long long i = 0;; ++i) {
            const int m = (int)(i % NM), s = (int)(i % kStrNCSlot);
            const int r = stream_wait_warp(a, bar(BI.cfull(s)), par(i, kStrNCSlot), i, s_end);
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile >= 0) {
                if (sw == 0 && lane == 0) trace_stamp(a, T.tile, 2);
                const uint32_t slot_s = smem_addr(cslot0 + (size_t)s * a.slot_bytes);
                for (int it = sw; it < n_steps; it += kStrNSum)
                    sum_pass_step(a, T, slot_s, it, NBT, M->abyte, M->blocksum, sarr(m), nullptr, lane);
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar(BI.bits(m)));
                mbar_arrive(bar(BI.cempty(s)));
            }
            if (T.tile < 0) break;
        }
    } else if (warp >= kStrMarks && warp < kStrMarks + kStrNMarks) {
        // ------------------------------------------------------------ windows, merge, aggregate, Q (alternate tiles)
        for (long long i = warp - kStrMarks;; i += kStrNMarks) {
            const int m = (int)(i % NM);
            const int r = stream_wait_warp(a, bar(BI.bits(m)), par(i, NM), i, s_end);
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) {
                if (lane == 0) mbar_arrive(bar(BI.agg(m)));
                break;
            }
            if (lane == 0) trace_stamp(a, T.tile, 3);
            const Agg agg = tile_bits<TW>(a, T, M->abyte, words(m), nullptr, lane);
            if (lane == 0) {
                M->agg = agg;
                if (T.tile > 0) publish(a.status, T.tile, false, agg, true);
                trace_stamp(a, T.tile, 4);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(BI.agg(m)));
            if (!skip_q) q_partial(a, T, M->blocksum, sarr(m), lane, 32);
        }
    } else if (warp >= kStrLook && warp < kStrLook + kStrNLook) {
        // ------------------------------------------------------------ decoupled look-back (tiles in turn)
        for (long long i = warp - kStrLook;; i += kStrNLook) {
            const int m = (int)(i % NM);
            const int r = stream_wait_warp(a, bar(BI.agg(m)), par(i, NM), i, s_end);
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) {
                if (lane == 0) mbar_arrive(bar(BI.excl(m)));
                break;
            }
            const Agg agg = M->agg;
            if (lane == 0) trace_stamp(a, T.tile, 5);
            unsigned lb_stats = 0;
            const Agg excl = T.tile > 0 ? look_back(a, T.tile, lane, &lb_stats) : agg_identity();
            if (lane == 0) {
                publish(a.status, T.tile, true, combine(excl, agg), true);
                M->excl = excl;
                trace_stamp(a, T.tile, 6);
                trace_value(a, T.tile, 14, lb_stats);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(BI.excl(m)));
        }
    } else if (warp == kStrLoader) {
        // ------------------------------------------------------------ marked steps -> step slots (from L2)
        const uint32_t qbox_bytes = (uint32_t)X * 2u * (uint32_t)kStrStep;
        const uint64_t pol = l2_policy_evict_first();  // last use of these lines
        long long g = 0;                                // steps loaded so far
        uint32_t pend_par = 0;                          // parity of the last load into each step slot
        uint32_t pending = 0;
        for (long long i = 0;; ++i) {
            const int m = (int)(i % NM);
            const int r = stream_wait_warp(a, bar(BI.excl(m)), par(i, NM), i, s_end);
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) break;
            if (skip_isl || M->agg.m == 0 || M->excl.poison) continue;
            uint32_t steps = marked_steps<TW>(M->wm, lane);
            const int c1 = (int)(((long long)T.f * a.n_calo + T.c) * X);
            bool ok = true;
            while (steps) {
                const int j = __ffs(steps) - 1;
                steps &= steps - 1u;
                const int q = (int)(g % kStrNQ);
                if (g >= kStrNQ &&
                    stream_wait_warp(a, bar(BI.qempty(q)), par_prev(g, kStrNQ), g, nullptr) != 1) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(bar(BI.qfull(q)), qbox_bytes);
                    tma_load_2d_hint(qslot0 + (size_t)q * qslot_bytes, &a.tmap_c, (int)T.t0 + kStrStep * j, c1,
                                     bar(BI.qfull(q)), pol);
                }
                pending |= 1u << q;
                pend_par = (pend_par & ~(1u << q)) | (par(g, kStrNQ) << q);
                ++g;
            }
            if (!ok) break;
            if (lane == 0) trace_stamp(a, T.tile, 12);
        }
        // copies still in flight land before this CTA may exit
        if (lane == 0)
            for (int q = 0; q < kStrNQ; ++q)
                if (pending & (1u << q)) mbar_wait_bounded(bar(BI.qfull(q)), (pend_par >> q) & 1u, kWaitLimitNs);
    } else if (warp >= kStrWriter0 && warp < kStrWriter0 + kStrNWriter) {
        // ------------------------------------------------------------ writers: rows of marked samples -> stage
        // Step g of the call goes to step slot g % kStrNQ; writer warp ww takes
        // the steps with g % kStrNWriter == ww, so each step slot has one owner.
        const int ww = warp - kStrWriter0;
        long long g = 0;
        for (long long i = 0;; ++i) {
            const int m = (int)(i % NM), o = (int)(i % NS);
            int r = stream_wait_warp(a, bar(BI.excl(m)), par(i, NM), i, s_end);
            if (r == 1 && i >= NS) r = stream_wait_warp(a, bar(BI.stage_free(o)), par_prev(i, NS), i, nullptr);
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile >= 0 && !skip_isl && M->agg.m > 0 && !M->excl.poison) {
                uint32_t steps = marked_steps<TW>(M->wm, lane);
                const int phase = (int)((M->excl.m * 2ll * X) & 15);
                const int nt = (int)(T.t_end - T.t0);
                unsigned char *stage = stage0 + (size_t)o * stage_bytes;
                bool ok = true;
                if (ww == 0 && lane == 0) trace_stamp(a, T.tile, 8);
                while (steps) {
                    const int j = __ffs(steps) - 1;
                    steps &= steps - 1u;
                    if (g % kStrNWriter == ww) {
                        const int q = (int)(g % kStrNQ);
                        if (stream_wait_warp(a, bar(BI.qfull(q)), par(g, kStrNQ), g, nullptr) != 1) {
                            ok = false;
                            break;
                        }
                        stage_step(a, smem_addr(qslot0 + (size_t)q * qslot_bytes), j, nt, M->wm, M->wmb, stage, phase,
                                   lane);
                        __syncwarp();
                        if (lane == 0) mbar_arrive(bar(BI.qempty(q)));
                    }
                    ++g;
                }
                if (!ok) break;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(BI.stage_full(o)));
            if (T.tile < 0) break;
        }
    } else {
        // ------------------------------------------------------------ store: stage -> pool, island records
        const long long rb = 2ll * X;
        bool any_store = false;
        for (long long i = 0;; ++i) {
            const int m = (int)(i % NM), o = (int)(i % NS);
            const int r = stream_wait_warp(a, bar(BI.stage_full(o)), par(i, NS), i, s_end);
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) break;
            const Agg agg = M->agg, excl = M->excl;
            bool rows = !skip_isl && agg.m > 0 && !excl.poison;
            if (rows && (a.flags & DAQ_DEBUG_CHECKS) && (excl.m < 0 || agg.m > T.t_end - T.t0)) {
                if (lane == 0) set_status_bit(a, DAQ_DEV_BAD_INDEX);  // more rows than the tile has samples
                rows = false;
            }
            if (lane == 0) trace_stamp(a, T.tile, 7);
            if (rows) {
                unsigned char *stage = stage0 + (size_t)o * stage_bytes;
                const long long gs = excl.m * rb;
                const int phase = (int)(gs & 15);
                long long ge = gs + agg.m * rb;
                const long long cap_b = a.pool_cap * rb;
                if (ge > cap_b) {
                    ge = cap_b;
                    if (lane == 0) set_status_bit(a, DAQ_DEV_POOL_OVERFLOW);
                }
                if (ge > gs) {
                    unsigned char *gp = reinterpret_cast<unsigned char *>(a.pool);
                    long long a16 = (gs + 15) & ~15ll, b16 = ge & ~15ll;
                    if (a16 > ge) a16 = ge;
                    if (b16 < a16) b16 = a16;
                    if (lane == 0 && b16 > a16) {
                        fence_proxy_async_smem();
                        bulk_s2g_hint(gp + a16, stage + phase + (a16 - gs), (uint32_t)(b16 - a16),
                                      l2_policy_evict_first());
                        bulk_commit();
                        any_store = true;
                    }
                    // unaligned ends: at most 7 two-byte stores on each side
                    const int n_head = (int)((a16 - gs) >> 1), n_tail = (int)((ge - b16) >> 1);
                    if (lane < n_head)
                        *reinterpret_cast<uint16_t *>(gp + gs + 2 * lane) =
                            *reinterpret_cast<const uint16_t *>(stage + phase + 2 * lane);
                    else if (lane >= 16 && lane < 16 + n_tail) {
                        const long long off = b16 + 2 * (lane - 16);
                        *reinterpret_cast<uint16_t *>(gp + off) =
                            *reinterpret_cast<const uint16_t *>(stage + phase + (off - gs));
                    }
                }
                if (lane == 0 && any_store) bulk_wait_read0();  // the stage has been read
                __syncwarp();
            }
            if (lane == 0) mbar_arrive(bar(BI.stage_free(o)));
            if (rows) write_headers<TW>(a, T, words(m), excl, lane);
            if (lane == 0 && T.tile == total - 1) write_counts(a, T.tile, combine(excl, agg));
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar(BI.meta_free(m)));
                trace_stamp(a, T.tile, 9);
            }
        }
        if (lane == 0 && any_store) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

}  // namespace daq
