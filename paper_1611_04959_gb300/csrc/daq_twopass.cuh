// Two-pass form of the per-fill processing (the default path), and its
// single-launch variant.
//
//   daq_count_kernel    every tile once, with its halo: crystal sums, pedestal
//                       subtraction, threshold, pre/post windows (the marks of
//                       the tile), Q-method partial bins; stores the tile's marks
//                       words and its aggregate (marked samples, island starts,
//                       trailing run).  No tile waits on another.
//   daq_scan_kernel     chained scan of the per-tile aggregates (blocks ordered
//                       by a ticket, decoupled look-back over earlier blocks):
//                       every tile's exclusive prefix (pool row and island
//                       index it starts at, marked run entering it) and the
//                       call's totals.
//   daq_compact_kernel  every tile again (tile proper only): the raw samples of
//                       its marked times are transposed into rows in shared
//                       memory at the phase of their global position, written
//                       with one bulk copy (plus unaligned ends), and the tile's
//                       island records are written.
//   daq_fused_kernel    the same three steps in one cooperative launch: count
//                       CTAs publish each tile's aggregate, one scanner CTA turns
//                       aggregates into prefixes in tile order, compact CTAs
//                       follow at most lag_tiles tiles behind the count CTAs, so
//                       the tile they re-read is still in L2.
#pragma once

#include "daq_steps.cuh"

namespace daq {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;  // tiles per scan thread
constexpr int kScanChunk = kScanThreads * kScanPer;

struct __align__(16) TileRec {
    int32_t m, s, tr, flags;  // flags: 1 continues (full), 2 mark before the tile, 4 mark after it
};
constexpr int32_t kRecValid = 0x100;  // single-launch form: the record has been published
constexpr int kRecStepShift = 16;     // flags bits 16..: the tile's 64-sample steps that hold a marked sample

// Bit j set when marks words 2j or 2j + 1 of the tile are non-zero (one warp,
// lane w holding word w; warp-uniform result).
template <int TW> __device__ __forceinline__ uint32_t marked_steps64(uint32_t Mt, int lane)
{
    constexpr int NWT = TW / 32;
    const uint32_t nz = __ballot_sync(kFull, lane < NWT && Mt != 0u);
    uint32_t steps = 0;
#pragma unroll
    for (int j = 0; j < (NWT + 1) / 2; ++j) steps |= ((nz >> (2 * j)) & 3u) ? (1u << j) : 0u;
    return steps;
}

struct __align__(16) TileExcl {
    long long m;  // pool rows before the tile
    int32_t s;    // islands starting before the tile
    int32_t tr;   // marked samples in the run entering the tile
};

__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_s2g_hint(void *dst, const void *src, uint32_t bytes, uint64_t policy)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                 "r"(smem_addr(src)), "r"(bytes), "l"(policy)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// ============================================================================ count pass
constexpr int kCountSumWarps = 8;
constexpr int kCountThreads = 32 * (kCountSumWarps + 2);  // + one marks/Q warp per tile slot (two slots)
constexpr int kPlanSmem = 64;                              // fills whose plan is cached in shared memory

// Per-fill plan (first tile, length) in shared memory when the batch has at
// most kPlanSmem fills; decode_tile then needs one global load (the pedestal).
struct PlanView {
    const long long *fts;
    const int32_t *lens;
};

__device__ __forceinline__ PlanView cache_plan(const KArgs &a, long long *fts_s, int32_t *lens_s, int tid, int nthr)
{
    if (a.n_fills > kPlanSmem) return PlanView{a.fill_tile_start, a.lens};
    for (int f = tid; f <= a.n_fills; f += nthr) fts_s[f] = a.fill_tile_start[f];
    for (int f = tid; f < a.n_fills; f += nthr) lens_s[f] = a.lens[f];
    return PlanView{fts_s, lens_s};
}

// Bounded mbarrier wait whose outcome is the same in every lane of the warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity)
{
    const bool ok = mbar_wait_bounded(bar, parity, kWaitLimitNs);
    return !__any_sync(kFull, !ok);
}

// As warp_wait, but also giving up once a CTA has flagged a timeout (the
// single-launch form, whose waits on other CTAs may run out).
__device__ __forceinline__ bool warp_wait_abortable(const KArgs &a, uint64_t *bar, uint32_t parity)
{
    bool ok = mbar_try_wait(bar, parity);
    if (!ok) {
        const uint64_t t0 = global_ns();
        for (uint32_t i = 1;; ++i) {
            if (mbar_try_wait(bar, parity)) {
                ok = true;
                break;
            }
            if ((i & 63u) == 0u && (aborted(a) || global_ns() - t0 > kWaitLimitNs)) break;
        }
    }
    return !__any_sync(kFull, !ok);
}

// Shared-memory layout of the count kernel with NS tile slots, in the order of
// the buffers.
template <int NS> struct CountSmemT {
    static size_t __host__ __device__ align16(size_t x) { return (x + 15) & ~size_t(15); }
    static size_t __host__ __device__ abyte(int slot_bytes) { return NS * (size_t)slot_bytes; }  // [NS][128]
    static size_t __host__ __device__ blocksum(int slot_bytes) { return abyte(slot_bytes) + 128 * NS; }  // [NS][TW/8]
    static size_t __host__ __device__ sarr(int slot_bytes, int tw)  // [NS][TW]
    {
        return blocksum(slot_bytes) + (size_t)NS * (size_t)(tw / 8) * 4;
    }
    static size_t __host__ __device__ tinfo(int slot_bytes, int tw, int need_sarr)
    {
        return align16(sarr(slot_bytes, tw) + (need_sarr ? (size_t)NS * 4 * (size_t)tw : 0));  // [2 NS]
    }
    static size_t __host__ __device__ fts(int slot_bytes, int tw, int need_sarr)
    {
        return tinfo(slot_bytes, tw, need_sarr) + 2 * NS * sizeof(TileInfo);  // [kPlanSmem + 1]
    }
    static size_t __host__ __device__ lens(int slot_bytes, int tw, int need_sarr)
    {
        return fts(slot_bytes, tw, need_sarr) + 8 * (kPlanSmem + 1);  // [kPlanSmem]
    }
    static size_t __host__ __device__ bars(int slot_bytes, int tw, int need_sarr)
    {
        return align16(lens(slot_bytes, tw, need_sarr) + 4 * kPlanSmem);  // full[NS], sums[NS], marks[NS]
    }
    static size_t __host__ __device__ total(int slot_bytes, int tw, int need_sarr)
    {
        return (bars(slot_bytes, tw, need_sarr) + 3 * NS * 8 + 127) & ~size_t(127);
    }
};
using CountSmem = CountSmemT<2>;
// Sum warps of the count kernel: 8 with two slots (two CTAs per SM), 16 with
// three (one CTA per SM keeps the SM's sum throughput).
template <int NS> __host__ __device__ constexpr int count_sum_warps() { return NS == 2 ? kCountSumWarps : 2 * kCountSumWarps; }
template <int NS> __host__ __device__ constexpr int count_threads() { return 32 * (count_sum_warps<NS>() + NS); }

// Progress counters of the single-launch form (workspace words).
__device__ __forceinline__ unsigned long long *scanned_ctr(const KArgs &a) { return a.fctr; }
__device__ __forceinline__ unsigned long long *compacted_ctr(const KArgs &a) { return a.fctr + 16; }

// Wait until *p >= v (acquire), giving up after the wait limit or when another
// CTA has flagged a timeout.  One thread.
__device__ __forceinline__ bool wait_counter_ge(const KArgs &a, const unsigned long long *p, unsigned long long v)
{
    if (ld_acquire_u64(p) >= v) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; ++i) {
        __nanosleep(64);
        if (ld_acquire_u64(p) >= v) return true;
        if (global_ns() - t0 > a.wait_ns) {
            set_status_bit(a, DAQ_DEV_TIMEOUT);
            return false;
        }
        if ((i & 63u) == 63u && aborted(a)) return false;
    }
}

// Eight sum warps turn a tile into threshold bits and block sums; marks warp
// s (one per buffer s = j mod NS) turns the bits of the CTA's tiles j = s,
// s + NS, ... into marks words and the tile aggregate and adds the tile's Q
// bins, while the sum warps go on with the next tile.  NS tile slots are
// loaded ahead by TMA.  Handoffs (per buffer): full (TMA landed), sums (8 sum warps done: the
// slot may be refilled and the bits read), marks (bits and block sums read:
// the buffer may be rewritten).  The CTA takes tiles first, first + G, ...
// kFused: a tile is loaded only while it is at most lag_tiles ahead of the
// tiles compacted, and its aggregate is published with a release store and a
// valid bit for the scanner.
// kHaloFree: the count pass loads the tile proper only (see complete_tile).
template <int TW, bool kFused, int NS = 2, bool kHaloFree = false>
__device__ __forceinline__ void count_role(const KArgs &a, unsigned char *smem, long long first, long long G)
{
    constexpr int NWT = TW / 32, NBT = TW / 8;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char *slot0 = smem;
    using SM = CountSmemT<NS>;
    constexpr int kThr = count_threads<NS>();
    constexpr int NSW = count_sum_warps<NS>();
    uint8_t *abyte0 = smem + SM::abyte(a.slot_bytes);
    int32_t *blocksum0 = reinterpret_cast<int32_t *>(smem + SM::blocksum(a.slot_bytes));
    int32_t *sarr0 = reinterpret_cast<int32_t *>(smem + SM::sarr(a.slot_bytes, TW));
    TileInfo *tinfo = reinterpret_cast<TileInfo *>(smem + SM::tinfo(a.slot_bytes, TW, a.need_sarr));
    TileInfo *tinfo_m = tinfo + NS;  // copies handed to the marks warps
    long long *fts_s = reinterpret_cast<long long *>(smem + SM::fts(a.slot_bytes, TW, a.need_sarr));
    int32_t *lens_s = reinterpret_cast<int32_t *>(smem + SM::lens(a.slot_bytes, TW, a.need_sarr));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SM::bars(a.slot_bytes, TW, a.need_sarr));
    uint64_t *full = bars, *sums = bars + NS, *mdone = bars + 2 * NS;

    for (int i = tid; i < 32 * NS; i += kThr) reinterpret_cast<uint32_t *>(abyte0)[i] = 0u;
    const PlanView plan = cache_plan(a, fts_s, lens_s, tid, kThr);

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full + s, 1);
            mbar_init(sums + s, NSW);
            mbar_init(mdone + s, 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const long long total = plan.fts[a.n_fills];
    const int n_steps = (a.ew + 63) / 64;
    constexpr int kSumThreads = 32 * NSW;

    uint32_t pend = 0, pend_par = 0;  // thread 0: slots with a load issued, parity of its phase
    auto start_load = [&](long long tile, int s) {  // thread 0
        if (kFused &&
            !wait_counter_ge(a, compacted_ctr(a), tile > a.lag_tiles ? (unsigned long long)(tile - a.lag_tiles) : 0ull))
            return;  // gave up (the flag is set): the sum warps stop at this slot
        TileInfo &T = tinfo[s];
        decode_tile<TW>(a, tile, T, plan.fts, plan.lens);
        trace_stamp(a, tile, 0);
        trace_value(a, tile, 10, sm_id());
        trace_value(a, tile, 11, TW);
        if (a.use_tma) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(full + s, tile_load_bytes(a));
            issue_tile_load(a, T, slot0 + (size_t)s * a.slot_bytes, full + s);
            if (kFused) {  // the single-launch form may stop early: loads in flight are waited for at exit
                pend |= 1u << s;
                pend_par = (pend_par & ~(1u << s)) | ((uint32_t)(((tile - first) / G / NS) & 1) << s);
            }
        }
        trace_stamp(a, tile, 1);
    };
    auto slot_wait = [&](uint64_t *bar, uint32_t parity) {
        return kFused ? warp_wait_abortable(a, bar, parity) : warp_wait(bar, parity);
    };

    if (warp < NSW) {
        if (tid == 0)
            for (int k = 0; k < NS; ++k)
                if (first + k * G < total) start_load(first + k * G, k);
        for (long long j = 0;; ++j) {
            const long long tile = first + j * G;
            if (tile >= total) break;
            const int s = (int)(j % NS);
            const uint32_t par = (uint32_t)((j / NS) & 1);
            unsigned char *slot = slot0 + (size_t)s * a.slot_bytes;
            if (a.use_tma) {
                if (!slot_wait(full + s, par)) {
                    if (lane == 0) set_status_bit(a, DAQ_DEV_TIMEOUT);
                    break;
                }
            } else {
                // sum warps only: the slot's previous tile (j - 2) is done and tinfo[s] is decoded
                asm volatile("bar.sync 1, %0;" ::"r"(kSumThreads) : "memory");
                plain_tile_load(a, tinfo[s], slot, tid, kSumThreads);
                asm volatile("bar.sync 1, %0;" ::"r"(kSumThreads) : "memory");
            }
            if (j >= NS && !slot_wait(mdone + s, par ^ 1u)) {
                if (lane == 0) set_status_bit(a, DAQ_DEV_TIMEOUT);
                break;
            }
            const TileInfo T = tinfo[s];
            if (tid == 0) {
                trace_stamp(a, T.tile, 2);
                tinfo_m[s] = T;
            }
            const uint32_t slot_s = smem_addr(slot);
            for (int it = warp; it < n_steps; it += NSW)
                sum_pass_step(a, T, slot_s, it, NBT, abyte0 + 128 * s, blocksum0 + NBT * s,
                              sarr0 + (a.need_sarr ? TW * s : 0), nullptr, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(sums + s);
            if (tid == 0) {
                trace_stamp(a, T.tile, 3);
                // slot s takes tile j + NS once every sum warp is done with tile j
                if (tile + NS * G < total) {
                    if (mbar_wait_bounded(sums + s, par, kWaitLimitNs)) {
                        if (a.use_tma) start_load(tile + NS * G, s);
                        else decode_tile<TW>(a, tile + NS * G, tinfo[s], plan.fts, plan.lens);
                    } else {
                        set_status_bit(a, DAQ_DEV_TIMEOUT);  // the other warps time out on tile j + 2
                    }
                }
            }
        }
        // a warp that stopped early leaves loads in flight: they land before
        // the CTA may exit (a slot's latest phase; immediate when consumed)
        if (kFused && tid == 0)
            for (int k = 0; k < NS; ++k)
                if (pend & (1u << k)) mbar_wait_bounded(full + k, (pend_par >> k) & 1u, kWaitLimitNs);
    } else if (warp < NSW + NS) {
        // ------------------------------------------------------------ marks, aggregate, Q bins of buffer s
        const int s = warp - NSW;
        const bool skip_q = (a.flags & DAQ_SKIP_Q) != 0;
        for (long long j = s;; j += NS) {
            const long long tile = first + j * G;
            if (tile >= total) break;
            if (!slot_wait(sums + s, (uint32_t)((j / NS) & 1))) {
                if (lane == 0) set_status_bit(a, DAQ_DEV_TIMEOUT);
                break;
            }
            const TileInfo T = tinfo_m[s];
            if (kHaloFree) {
                // internal marks of the tile and its first / last crossing; the
                // scan adds the marks that crossings of neighbouring tiles reach
                const uint32_t A = lane < NWT ? reinterpret_cast<const uint32_t *>(abyte0 + 128 * s)[lane] : 0u;
                const int nt = (int)(T.t_end - T.t0);
                const uint32_t Mi = marks_word(a, A, lane) & range_mask(32ll * lane, 0, nt);
                const unsigned fb = (unsigned)__reduce_min_sync(kFull, A ? (unsigned)(32 * lane + __ffs(A) - 1) : 0xffffffffu);
                const int lb = (int)__reduce_max_sync(kFull, A ? (unsigned)(32 * lane + 32 - __clz(A)) : 0u) - 1;
                if (lane < NWT) a.marks[T.tile * NWT + lane] = Mi;
                if (lane == 0)  // first and last crossing (-1: none), tile within its calorimeter-fill, fill length
                    *reinterpret_cast<int4 *>(&a.status[T.tile]) =
                        make_int4(fb != 0xffffffffu ? (int)(T.t0 + fb) : -1, lb >= 0 ? (int)(T.t0 + lb) : -1,
                                  (int)(T.t0 / TW), (int)T.len);
                if (!skip_q) q_partial(a, T, blocksum0 + NBT * s, sarr0 + (a.need_sarr ? TW * s : 0), lane, 32);
                __syncwarp();
                if (lane == 0) mbar_arrive(mdone + s);
                continue;
            }
            unsigned edges;
            const uint32_t Mt = tile_marks<TW>(a, T, abyte0 + 128 * s, &edges, lane);
            const Agg agg = agg_from_marks<TW>(Mt, edges & 1u, (int)(T.t_end - T.t0), lane);
            const uint32_t steps = marked_steps64<TW>(Mt, lane);
            if (lane < NWT) a.marks[T.tile * NWT + lane] = Mt;
            if (kFused) {
                __threadfence();
                __syncwarp();
            }
            if (lane == 0) {
                TileRec r;
                r.m = (int32_t)agg.m;
                r.s = (int32_t)agg.s;
                r.tr = (int32_t)agg.tr;
                r.flags = (agg.full ? 1 : 0) | (int)((edges & 1u) << 1) | (int)((edges >> 1) << 2) |
                          (int)(steps << kRecStepShift);
                if (kFused) {
                    // marks words first, then the record with its valid bit (release)
                    __threadfence();
                    const unsigned long long lo = (unsigned long long)(uint32_t)r.m | ((unsigned long long)(uint32_t)r.s << 32);
                    const unsigned long long hi =
                        (unsigned long long)(uint32_t)r.tr | ((unsigned long long)(uint32_t)(r.flags | kRecValid) << 32);
                    st_release_b128(reinterpret_cast<TileRec *>(a.recs) + T.tile, lo, hi);
                } else {
                    reinterpret_cast<TileRec *>(a.recs)[T.tile] = r;
                }
                trace_stamp(a, T.tile, 4);
            }
            if (!skip_q) q_partial(a, T, blocksum0 + NBT * s, sarr0 + (a.need_sarr ? TW * s : 0), lane, 32);
            __syncwarp();
            if (lane == 0) mbar_arrive(mdone + s);
        }
    }
}

// NS = 2: two CTAs per SM; NS = 3: one CTA per SM with 16 sum warps, for
// extended tiles too wide for two CTAs' slots to fit.  HF: halo-free.
template <int TW, int NS, bool HF>
__global__ void __launch_bounds__(count_threads<NS>(), NS == 2 ? 2 : 1) daq_count_kernel(const __grid_constant__ KArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();     // the prepare kernel's plan, pedestals and resets
    pdl_trigger();  // the scan may be scheduled as CTAs finish
    count_role<TW, false, NS, HF>(a, smem, blockIdx.x, gridDim.x);
}

// ============================================================================ scan of the aggregates
__device__ __forceinline__ Agg rec_agg(const TileRec &r)
{
    Agg g;
    g.m = r.m;
    g.s = r.s;
    g.tr = r.tr;
    g.full = r.flags & 1;
    g.poison = 0;
    return g;
}

// Ordered inclusive scan across a block of 256 threads (v: this thread's value,
// later threads hold later tiles).  Returns the inclusive value; *block_total
// gets the combination over all threads.
__device__ __forceinline__ Agg block_scan_incl(Agg v, Agg *warp_tot, Agg *block_total)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const Agg o = shfl_up_agg(v, d);
        if (lane >= d) v = combine(o, v);
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (tid == 0) {
        Agg acc = warp_tot[0];
        for (int w = 1; w < kScanThreads / 32; ++w) {
            acc = combine(acc, warp_tot[w]);
            warp_tot[w] = acc;  // inclusive over warps 0..w
        }
    }
    __syncthreads();
    if (warp > 0) v = combine(warp_tot[warp - 1], v);
    *block_total = warp_tot[kScanThreads / 32 - 1];
    return v;
}

// Halo-free count pass: tile j's marks from its internal marks and the
// threshold crossings of the neighbouring tiles of its calorimeter-fill (a
// crossing at u marks [u - pre, u + post]: only the last crossing at most post
// before the tile and the first at most pre after it can reach it).  Stores
// the completed marks words and returns the tile's record: aggregate, marks of
// the samples just before and after the tile, marked 64-sample steps.
template <int TW> __device__ TileRec complete_tile(const KArgs &a, long long j)
{
    constexpr int NWT = TW / 32;
    constexpr int kReach = 4;  // neighbouring tiles read at once on each side
    const int4 own = *reinterpret_cast<const int4 *>(&a.status[j]);
    const long long t0 = (long long)own.z * TW, len = own.w;
    const long long t_end = t0 + TW < len ? t0 + TW : len;
    const long long cf0 = j - own.z, cf1 = cf0 + (len + TW - 1) / TW;  // tiles of the calorimeter-fill
    const int nt = (int)(t_end - t0);
    const long long kNone = 1ll << 40;
    long long Lp = -kNone, Fn = kNone;  // last crossing before the tile, first after it
    const int kb = a.post / TW + 1, kf = a.pre / TW + 1;  // tiles a window reaches
    for (int k0 = 1; k0 <= kb && Lp == -kNone; k0 += kReach) {
        int l[kReach];
#pragma unroll
        for (int u = 0; u < kReach; ++u) {
            const long long k = j - (k0 + u);
            l[u] = (k0 + u <= kb && k >= cf0) ? reinterpret_cast<const int2 *>(&a.status[k])->y : -1;
        }
#pragma unroll
        for (int u = 0; u < kReach; ++u)
            if (Lp == -kNone && l[u] >= 0) Lp = l[u];
    }
    for (int k0 = 1; k0 <= kf && Fn == kNone; k0 += kReach) {
        int f[kReach];
#pragma unroll
        for (int u = 0; u < kReach; ++u) {
            const long long k = j + (k0 + u);
            f[u] = (k0 + u <= kf && k < cf1) ? reinterpret_cast<const int2 *>(&a.status[k])->x : -1;
        }
#pragma unroll
        for (int u = 0; u < kReach; ++u)
            if (Fn == kNone && f[u] >= 0) Fn = f[u];
    }
    const long long from_before = Lp + a.post - t0;  // tile columns [0, from_before] are marked from before
    const long long from_after = Fn - a.pre - t0;    // and [from_after, nt) from after
    const long long first_at = own.x >= 0 ? own.x : Fn, last_at = own.y >= 0 ? own.y : Lp;
    const uint32_t m_prev = t0 > 0 && (Lp >= t0 - 1 - a.post || first_at <= t0 - 1 + a.pre);
    const uint32_t m_next = t_end < len && (last_at >= t_end - a.post || Fn <= t_end + a.pre);
    uint32_t *mw = a.marks + j * NWT;
    uint32_t W[NWT];
#pragma unroll
    for (int w = 0; w < NWT; ++w) W[w] = mw[w];
    int m = 0, st = 0, lz = -1;
    uint32_t steps = 0, below = m_prev;
#pragma unroll
    for (int w = 0; w < NWT; ++w) {
        const long long b = 32ll * w;
        const uint32_t add = range_mask(b, 0, from_before + 1) | range_mask(b, from_after, nt);
        const uint32_t Wf = (W[w] | add) & range_mask(b, 0, nt);
        if (Wf != W[w]) mw[w] = Wf;
        m += __popc(Wf);
        st += __popc(Wf & ~((Wf << 1) | below));
        below = Wf >> 31;
        const uint32_t zeros = ~Wf & range_mask(b, 0, nt);
        if (zeros) lz = 32 * w + 31 - __clz(zeros);
        if (Wf) steps |= 1u << (w >> 1);
    }
    TileRec r;
    r.m = m;
    r.s = st;
    r.tr = nt - 1 - lz;
    r.flags = ((lz < 0 && m_prev) ? 1 : 0) | (int)(m_prev << 1) | (int)(m_next << 2) | (int)(steps << kRecStepShift);
    return r;
}

// Single-launch chained scan: blocks take chunks of kScanChunk tiles in ticket
// order (so every chunk's predecessors are running or done); each reduces its chunk,
// publishes the aggregate, looks back over earlier chunks' published states
// for its exclusive prefix (one warp), publishes its inclusive prefix and
// writes every tile's exclusive prefix.  After a halo-free count pass (HF) it
// first completes its tiles' marks and records.
template <int TW, bool HF>
__global__ void __launch_bounds__(kScanThreads) daq_scan_kernel(const __grid_constant__ KArgs a)
{
    pdl_wait();  // every tile's record
    pdl_trigger();
    __shared__ Agg warp_tot[kScanThreads / 32];
    __shared__ Agg s_incl[kScanThreads];
    __shared__ Agg s_prefix;
    __shared__ long long s_chunk;
    if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(a.scan_ticket, 1u);
    __syncthreads();
    const long long chunk = s_chunk;
    const long long total = a.fill_tile_start[a.n_fills];
    const long long chunk0 = chunk * kScanChunk;
    if (chunk0 >= total) return;  // grids are sized for the largest tile count
    const long long base = chunk0 + (long long)threadIdx.x * kScanPer;
    TileRec *recs = reinterpret_cast<TileRec *>(a.recs);
    TileRec r[kScanPer];
    Agg v = agg_identity();
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i >= total) r[i] = TileRec{0, 0, 0, 1};
        else if (HF) {
            r[i] = complete_tile<TW>(a, base + i);
            recs[base + i] = r[i];  // the compact pass reads the completed record and marks
        } else r[i] = recs[base + i];
        v = combine(v, rec_agg(r[i]));
    }
    Agg blk_tot;
    s_incl[threadIdx.x] = block_scan_incl(v, warp_tot, &blk_tot);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        Agg ex = agg_identity();
        if (chunk > 0) {
            if (lane == 0) publish(a.scan_status, chunk, false, blk_tot, true);
            ex = look_back_in(a, a.scan_status, chunk, lane);
        }
        if (lane == 0) {
            publish(a.scan_status, chunk, true, combine(ex, blk_tot), true);
            s_prefix = ex;
        }
    }
    __syncthreads();
    const Agg prefix = s_prefix;
    Agg ex = threadIdx.x == 0 ? prefix : combine(prefix, s_incl[threadIdx.x - 1]);
    TileExcl *out = reinterpret_cast<TileExcl *>(a.excl);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < total) {
            TileExcl e;
            e.m = ex.m;
            e.s = (int32_t)ex.s;
            e.tr = (int32_t)ex.tr;
            out[base + i] = e;
            if (base + i == total - 1) write_counts(a, total - 1, combine(ex, rec_agg(r[i])));
        }
        ex = combine(ex, rec_agg(r[i]));
    }
}

// ============================================================================ compact pass
// Stage the rows of the marked samples of 64 tile columns (one warp): lane L
// owns columns c = 64 it + 2L, c + 1 of the tile proper; a marked sample's row
// goes to byte phase + r * 2X of the stage, r = its rank among the tile's
// marked samples.
__device__ __forceinline__ void compact_step(const KArgs &a, uint32_t slot_s, int it, int nt, const uint32_t *wm,
                                             const int32_t *wmb, unsigned char *stage, int phase, int lane)
{
    const int X = a.n_xtal;
    const int c = 64 * it + 2 * lane;
    const int w = c >> 5, bit = c & 31;
    const uint32_t mw = c < nt ? wm[w] : 0u;
    const uint32_t m0 = (mw >> bit) & 1u, m1 = c + 1 < nt ? (mw >> (bit + 1)) & 1u : 0u;
    if (!__any_sync(kFull, m0 | m1)) return;
    if (!(m0 | m1)) return;
    const int r0 = wmb[w] + __popc(mw & ((1u << bit) - 1u));
    const int r1 = r0 + (int)m0;
    const int k = (c >= a.boxw_b) + (c >= 2 * a.boxw_b) + (c >= 3 * a.boxw_b) + (c >= 4 * a.boxw_b);
    const uint32_t base = slot_s + (uint32_t)(k * a.box_stride_b + 2 * (c - k * a.boxw_b));
    unsigned char *row0 = stage + phase + (size_t)r0 * 2 * X, *row1 = stage + phase + (size_t)r1 * 2 * X;
    if (!(X & 1)) {
#pragma unroll 3
        for (int x = 0; x < X; x += 2) {
            const uint32_t w0 = lds_u32(base + (uint32_t)(x * a.rs_b));
            const uint32_t w1 = lds_u32(base + (uint32_t)((x + 1) * a.rs_b));
            if (m0) *reinterpret_cast<uint32_t *>(row0 + 2 * x) = __byte_perm(w0, w1, 0x5410);
            if (m1) *reinterpret_cast<uint32_t *>(row1 + 2 * x) = __byte_perm(w0, w1, 0x7632);
        }
    } else {
        for (int x = 0; x < X; ++x) {
            const uint32_t w0 = lds_u32(base + (uint32_t)(x * a.rs_b));
            if (m0) *reinterpret_cast<uint16_t *>(row0 + 2 * x) = (uint16_t)(w0 & 0xffffu);
            if (m1) *reinterpret_cast<uint16_t *>(row1 + 2 * x) = (uint16_t)(w0 >> 16);
        }
    }
}

// Load the boxes of the tile proper whose bit is set in `boxes` (one thread;
// the caller armed `bar` for their bytes).
__device__ __forceinline__ void issue_tile_load_b(const KArgs &a, const TileInfo &T, unsigned char *slot,
                                                  uint64_t *bar, uint32_t boxes)
{
    const int c0 = (int)T.t0;
    const int c1 = (int)(((long long)T.f * a.n_calo + T.c) * a.n_xtal);
    const bool last_use = a.mode == kModeFused || a.mode == kModeStream;
    const uint64_t pol = l2_policy_evict_first();
    for (int k = 0; k < a.nbox_b; ++k) {
        if (!((boxes >> k) & 1u)) continue;
        if (last_use) tma_load_2d_hint(slot + (size_t)k * a.box_stride_b, &a.tmap_b, c0 + k * a.boxw_b, c1, bar, pol);
        else tma_load_2d(slot + (size_t)k * a.box_stride_b, &a.tmap_b, c0 + k * a.boxw_b, c1, bar);
    }
}

__device__ __forceinline__ void plain_tile_load_b(const KArgs &a, const TileInfo &T, unsigned char *slot, int tid,
                                                  int nthr)
{
    const int X = a.n_xtal, W = a.nbox_b * a.boxw_b;
    const long long cf = (long long)T.f * a.n_calo + T.c;
    const int16_t *rows = a.samples + cf * X * a.n_samples;
    for (int i = tid; i < X * W; i += nthr) {
        const int x = i / W, c = i - x * W;
        const int k = c / a.boxw_b, col = c - k * a.boxw_b;
        const long long t = T.t0 + c;
        int16_t v = 0;
        if (t < a.n_samples) v = rows[(long long)x * a.n_samples + t];
        *reinterpret_cast<int16_t *>(slot + (size_t)k * a.box_stride_b + (size_t)x * a.rs_b + 2 * col) = v;
    }
}

// One tile slot: the next tile's load is issued as soon as the current tile's
// rows are staged, so it lands while the pool rows and island records of the
// current tile are written; the marks, record and prefix of the next tile are
// loaded into registers at the same point.  The CTA takes tiles first, first +
// G, ...; any block size that is a multiple of 32 and >= 128.
// kSparse (DAQ_SPARSE): tiles without a marked sample (no rows, no island
// starts: nothing to write) are passed over.  With the next tile's inputs
// warp 0 also reads the record of the tile after it; when that tile has no
// marked sample, warp 0 reads the records of the 32 tiles after it at once,
// while the current tile's load lands, and leaves the first with one in
// shared memory.  The default form keeps a fixed stride: on fills where
// nearly every tile holds a marked sample the extra steps cost 0.5-1%.
// kFused: a tile's marks, record and prefix are read once the scanner has
// passed it (L1-bypassing loads: other CTAs wrote them during this launch), and
// each tile staged is counted in the compacted counter.
template <int TW, bool kFused, bool kSparse = false>
__device__ __forceinline__ void compact_role(const KArgs &a, unsigned char *smem, long long first, long long G)
{
    constexpr int NWT = TW / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarps = nthr >> 5;
    const int X = a.n_xtal;
    unsigned char *slot = smem;
    unsigned char *stage = slot + a.slot_bytes_b;  // TW rows of 2X bytes, 16-byte phase, + 32
    const int stage_bytes = ((TW * 2 * X + 32) + 15) & ~15;
    uint32_t *wm = reinterpret_cast<uint32_t *>(stage + stage_bytes);
    TileWords W{wm, wm + NWT, wm + 2 * NWT, reinterpret_cast<int32_t *>(wm + 3 * NWT),
                reinterpret_cast<int32_t *>(wm + 4 * NWT), reinterpret_cast<int32_t *>(wm + 5 * NWT)};
    TileInfo *tinfo = reinterpret_cast<TileInfo *>((reinterpret_cast<uintptr_t>(wm + 6 * NWT) + 15) & ~uintptr_t(15));
    Agg *s_ex = reinterpret_cast<Agg *>(tinfo + 1);
    Agg *s_agg = s_ex + 1;
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_agg + 1);
    long long *fts_s = reinterpret_cast<long long *>(bar + 1);             // [kPlanSmem + 1]
    int32_t *lens_s = reinterpret_cast<int32_t *>(fts_s + kPlanSmem + 1);  // [kPlanSmem]
    uint32_t *s_boxes = reinterpret_cast<uint32_t *>(lens_s + kPlanSmem);  // boxes of the CTA's next tile
    // kSparse: the CTA's next tile, when tile + G holds no marked sample
    long long *s_next = reinterpret_cast<long long *>((reinterpret_cast<uintptr_t>(s_boxes + 1) + 7) & ~uintptr_t(7));
    const PlanView plan = cache_plan(a, fts_s, lens_s, tid, nthr);
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const long long total = plan.fts[a.n_fills];
    const TileRec *recs = reinterpret_cast<const TileRec *>(a.recs);
    const TileExcl *exs = reinterpret_cast<const TileExcl *>(a.excl);
    const uint32_t one_box = (uint32_t)X * (uint32_t)a.rs_b;
    const uint32_t all_boxes = (1u << a.nbox_b) - 1u;
    // Boxes of a tile to load: those covering a 64-sample step its count record
    // marks (box k holds columns [k boxw, (k + 1) boxw)); the single-launch
    // form's records may not be published yet: all.
    auto flags_of = [&](long long tile) -> uint32_t {
        return (kFused || tile >= total) ? ~0u : (uint32_t)recs[tile].flags;
    };
    auto boxes_of = [&](uint32_t flags) -> uint32_t {
        if (flags == ~0u) return all_boxes;
        const uint32_t steps = flags >> kRecStepShift;
        uint32_t boxes = 0;
        for (int k = 0; k < a.nbox_b; ++k) {
            const int s0 = (k * a.boxw_b) >> 6, s1 = ((k + 1) * a.boxw_b - 1) >> 6;
            const uint32_t m = (s1 >= 31 ? 0xffffffffu : ((2u << s1) - 1u)) & ~((1u << s0) - 1u);
            if (steps & m) boxes |= 1u << k;
        }
        return boxes;
    };
    // kSparse, warp 0: the first of tiles t, t + G, ... that holds a marked
    // sample (total if none) and its record flags, in every lane
    auto find_next = [&](long long t, long long &nt, uint32_t &fl) {
        for (;; t += 32 * G) {
            if (t >= total) {
                nt = total;
                fl = 0u;
                return;
            }
            const long long u = t + lane * G;
            int m = 0;
            uint32_t f = 0u;
            if (u < total) {
                const int4 rv = *reinterpret_cast<const int4 *>(recs + u);
                m = rv.x;
                f = (uint32_t)rv.w;
            }
            const uint32_t stop = __ballot_sync(kFull, u >= total || m != 0);
            if (stop) {
                const int k = __ffs(stop) - 1;
                const long long v = t + (long long)k * G;
                nt = v < total ? v : total;
                fl = __shfl_sync(kFull, f, k);
                return;
            }
        }
    };
    auto start_load = [&](long long tile, uint32_t boxes) {  // one thread
        // no pedestal sum: the compact pass does not use it, and its load would
        // delay the bulk copy
        decode_tile<TW>(a, tile, *tinfo, plan.fts, plan.lens, false);
        trace_stamp(a, tile, 5);
        if (a.use_tma) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, (uint32_t)__popc(boxes) * one_box);
            issue_tile_load_b(a, *tinfo, slot, bar, boxes);
        }
    };

    // warp 0's inputs of the next tile, in registers, and (lane 0) the record
    // flags of the tile after it (kSparse: and its marked samples); false if
    // the wait gave up
    auto load_inputs = [&](long long tile, uint32_t &Mt, TileRec &r, TileExcl &e, int &m2, uint32_t &fl2) -> bool {
        if constexpr (kSparse) {
            m2 = 1;
            fl2 = 0u;
            if (lane == 0 && tile + G < total) {
                const int4 rv = *reinterpret_cast<const int4 *>(recs + tile + G);
                m2 = rv.x;
                fl2 = (uint32_t)rv.w;
            }
        } else {
            fl2 = lane == 0 ? flags_of(tile + G) : 0u;
        }
        if (kFused) {
            int ok = 1;
            if (lane == 0) ok = wait_counter_ge(a, scanned_ctr(a), (unsigned long long)tile + 1ull) ? 1 : 0;
            if (!__shfl_sync(kFull, ok, 0)) return false;
            Mt = lane < NWT ? __ldcg(a.marks + tile * NWT + lane) : 0u;
            const int4 rv = __ldcg(reinterpret_cast<const int4 *>(recs + tile));
            r = TileRec{rv.x, rv.y, rv.z, rv.w};
            const longlong2 ev = __ldcg(reinterpret_cast<const longlong2 *>(exs + tile));
            e.m = ev.x;
            e.s = (int32_t)(ev.y & 0xffffffffll);
            e.tr = (int32_t)(ev.y >> 32);
        } else {
            Mt = lane < NWT ? a.marks[tile * NWT + lane] : 0u;
            r = recs[tile];
            e = exs[tile];
        }
        return true;
    };

    uint32_t phase_bit = 0;
    bool store_pending = false;
    bool load_pending = false;  // thread 32 (single-launch form): a load issued that no thread has waited for
    uint32_t nMt = 0, nfl2 = 0;
    int nm2 = 1;  // kSparse, lane 0 of warp 0: marked samples of the next tile + G
    TileRec nr{0, 0, 0, 0};
    TileExcl ne{0, 0, 0};
    int in_ok = 1;
    if (first < total) {
        if (tid == 32) {
            start_load(first, boxes_of(flags_of(first)));
            load_pending = kFused;
        }
        if (warp == 0) in_ok = load_inputs(first, nMt, nr, ne, nm2, nfl2) ? 1 : 0;
    }
    for (long long tile = first; tile < total;) {
        int moved = 0;  // kSparse, warp 0: the next tile is not tile + G (it is in s_next)
        if (__syncthreads_or(!in_ok)) break;  // tinfo holds this tile; warp 0 has its inputs
        const TileInfo T = *tinfo;
        if (!a.use_tma) plain_tile_load_b(a, T, slot, tid, nthr);
        if (warp == 0) {
            const Agg g = words_from_marks<TW>(nMt, (nr.flags >> 1) & 1, (nr.flags >> 2) & 1,
                                               (int)(T.t_end - T.t0), W, nullptr, lane);
            uint32_t fl = nfl2;
            if constexpr (kSparse) {
                if (tile + G < total && __shfl_sync(kFull, nm2, 0) == 0) {
                    // tile + G holds no marked sample: find the CTA's next one
                    long long nt;
                    find_next(tile + 2 * G, nt, fl);
                    moved = 1;
                    if (lane == 0) *s_next = nt;
                }
            }
            if (lane == 0) {
                *s_boxes = boxes_of(fl);  // read with this tile's inputs; the next load uses it
                Agg ex;
                ex.m = ne.m;
                ex.s = ne.s;
                ex.tr = ne.tr;
                ex.full = 0;
                ex.poison = 0;
                *s_ex = ex;
                *s_agg = g;
                if (store_pending) {  // the stage is free once the last bulk store has read it
                    bulk_wait_read0();
                    store_pending = false;
                }
            }
        }
        if (a.use_tma) {
            const bool ok = mbar_wait_bounded(bar, phase_bit, kWaitLimitNs);
            if (ok) load_pending = false;
            phase_bit ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) set_status_bit(a, DAQ_DEV_TIMEOUT);
                break;
            }
        } else {
            __syncthreads();
        }
        const Agg ex = *s_ex, agg = *s_agg;
        if (tid == 0) trace_stamp(a, tile, 6);
        const long long rb = 2ll * X;
        const long long gs = ex.m * rb;
        const int phase = (int)(gs & 15);
        const int nt = (int)(T.t_end - T.t0);
        for (int it = warp; it < (nt + 63) / 64; it += nwarps)
            compact_step(a, smem_addr(slot), it, nt, W.m, W.mb, stage, phase, lane);
        // rows staged; the slot is free
        long long next = tile + G;
        if constexpr (kSparse) {
            if (__syncthreads_or(tid == 0 && moved)) next = *s_next;
        } else {
            __syncthreads();
        }
        if (kFused && tid == 0) atomicAdd(compacted_ctr(a), 1ull);
        if (next < total) {
            if (tid == 32) {
                start_load(next, *s_boxes);
                load_pending = kFused && a.use_tma;  // the single-launch form may stop before waiting for it
            }
            if (warp == 0) in_ok = load_inputs(next, nMt, nr, ne, nm2, nfl2) ? 1 : 0;
        }
        if (tid == 0) trace_stamp(a, tile, 7);
        // rows [ex.m, ex.m + agg.m) <- stage bytes [phase, phase + agg.m * 2X)
        long long ge = gs + agg.m * rb;
        if ((a.flags & DAQ_DEBUG_CHECKS) && (ex.m < 0 || agg.m < 0 || agg.m > nt)) {
            // the stage holds at most the tile's samples
            if (tid == 0) set_status_bit(a, DAQ_DEV_BAD_INDEX);
            ge = gs;
        }
        const long long cap_b = a.pool_cap * rb;
        if (ge > cap_b) {
            ge = cap_b;
            if (tid == 0) set_status_bit(a, DAQ_DEV_POOL_OVERFLOW);
        }
        if (ge > gs) {
            unsigned char *g = reinterpret_cast<unsigned char *>(a.pool);
            long long a16 = (gs + 15) & ~15ll, b16 = ge & ~15ll;
            if (a16 > ge) a16 = ge;
            if (b16 < a16) b16 = a16;
            // stage offset of global byte x is phase + (x - gs); a16 maps to a multiple of 16
            if (tid == 0 && b16 > a16) {
                fence_proxy_async_smem();
                if (kFused)  // pool rows are not read again here: let them leave L2 first
                    bulk_s2g_hint(g + a16, stage + phase + (a16 - gs), (uint32_t)(b16 - a16), l2_policy_evict_first());
                else
                    bulk_s2g(g + a16, stage + phase + (a16 - gs), (uint32_t)(b16 - a16));
                bulk_commit();
                store_pending = true;
            }
            const int n_head = (int)((a16 - gs) >> 1), n_tail = (int)((ge - b16) >> 1);
            if (tid >= 64 && tid < 64 + n_head)
                *reinterpret_cast<uint16_t *>(g + gs + 2 * (tid - 64)) =
                    *reinterpret_cast<const uint16_t *>(stage + phase + 2 * (tid - 64));
            else if (tid >= 96 && tid < 96 + n_tail) {
                const long long o = b16 + 2 * (tid - 96);
                *reinterpret_cast<uint16_t *>(g + o) = *reinterpret_cast<const uint16_t *>(stage + phase + (o - gs));
            }
        }
        if (warp == 0) write_headers<TW>(a, T, W, ex, lane);
        if (tid == 0) trace_stamp(a, tile, 9);
        tile = next;
    }
    if (tid == 0 && store_pending) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (tid == 32 && load_pending) mbar_wait_bounded(bar, phase_bit, kWaitLimitNs);  // left early: let it land
}

template <int TW, bool kSparse>
__global__ void __launch_bounds__(256, 2) daq_compact_kernel(const __grid_constant__ KArgs a)
{
    pdl_wait();                // every tile's prefix
    if (aborted(a)) return;    // the scan gave up: its prefixes are incomplete
    extern __shared__ __align__(128) unsigned char smem[];
    compact_role<TW, false, kSparse>(a, smem, blockIdx.x, gridDim.x);
}

// ============================================================================ single-launch form
// Scanner: tiles in order, blockDim.x at a time.  Each thread waits for its
// tile's published record, the block scans the aggregates (carrying the
// prefix of everything before), writes every tile's exclusive prefix, then
// releases the scanned counter.
__device__ __forceinline__ void scan_role(const KArgs &a)
{
    __shared__ Agg s_wtot[32];
    __shared__ Agg s_carry;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const long long total = a.fill_tile_start[a.n_fills];
    TileExcl *out = reinterpret_cast<TileExcl *>(a.excl);
    const TileRec *recs = reinterpret_cast<const TileRec *>(a.recs);
    if (tid == 0) {
        s_carry = agg_identity();
        s_fail = 0;
    }
    __syncthreads();
    for (long long base = 0; base < total; base += blockDim.x) {
        const long long t = base + tid;
        Agg v = agg_identity();
        TileRec r{0, 0, 0, 1};
        if (t < total) {
            unsigned long long lo = 0, hi = 0;
            ld_acquire_b128(recs + t, lo, hi);
            const uint64_t t0 = global_ns();
            for (uint32_t i = 0; !((hi >> 32) & (unsigned long long)kRecValid); ++i) {
                __nanosleep(128);
                ld_acquire_b128(recs + t, lo, hi);
                if (global_ns() - t0 > a.wait_ns || ((i & 63u) == 63u && aborted(a))) {
                    s_fail = 1;
                    break;
                }
            }
            r = TileRec{(int32_t)(lo & 0xffffffffull), (int32_t)(lo >> 32), (int32_t)(hi & 0xffffffffull),
                        (int32_t)(hi >> 32)};
            v = rec_agg(r);
        }
        // inclusive scan of v across the block
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Agg o = shfl_up_agg(v, d);
            if (lane >= d) v = combine(o, v);
        }
        if (lane == 31) s_wtot[warp] = v;
        __syncthreads();
        if (s_fail) {
            if (tid == 0) set_status_bit(a, DAQ_DEV_TIMEOUT);
            return;
        }
        Agg pre = s_carry;
        for (int w = 0; w < warp; ++w) pre = combine(pre, s_wtot[w]);
        const Agg incl = combine(pre, v);
        const Agg vprev = shfl_up_agg(v, 1);  // warp-inclusive value of the previous lane
        if (t < total) {
            const Agg ex = lane == 0 ? pre : combine(pre, vprev);
            TileExcl e;
            e.m = ex.m;
            e.s = (int32_t)ex.s;
            e.tr = (int32_t)ex.tr;
            out[t] = e;
            if (t == total - 1) write_counts(a, t, incl);
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) {
            Agg c = s_carry;
            for (int w = 0; w < nw; ++w) c = combine(c, s_wtot[w]);
            s_carry = c;
            __threadfence();
            const long long done = base + blockDim.x < total ? base + blockDim.x : total;
            st_release_u64(scanned_ctr(a), (unsigned long long)done);
        }
        __syncthreads();
    }
}

// Roles by block: 0 scanner, [1, G/2) compact, [G/2, G) count.  Launched
// cooperatively, so every CTA is resident and the waits between roles end.
template <int TW>
__global__ void __launch_bounds__(kCountThreads, 2) daq_fused_kernel(const __grid_constant__ KArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const long long G = gridDim.x, half = G / 2;
    if (blockIdx.x == 0) scan_role(a);
    else if (blockIdx.x < half) compact_role<TW, true>(a, smem, blockIdx.x - 1, half - 1);
    else count_role<TW, true>(a, smem, blockIdx.x - half, G - half);
}

}  // namespace daq
