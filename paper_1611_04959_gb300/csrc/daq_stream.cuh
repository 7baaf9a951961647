// Streaming single-pass form (daq_params.grid = -5): every sample is read from
// HBM once, and the compaction re-reads each tile from L2.
//
// One persistent CTA per SM; warps have fixed roles and hand tiles to each
// other through mbarriers over a ring of kStrNMeta tile records in shared
// memory:
//
//   producer     takes a ticket (tiles run in ticket order), decodes the tile
//                and asks L2 to prefetch its extended rows;
//   count warps  crystal sums straight from global memory into registers: a
//                lane owns 8 consecutive samples of a 256-sample strip and adds
//                the 54 crystals' 16-byte words with dp2a (Table 2 rows 1, 6),
//                subtracts the summed pedestals and tests the threshold (row 2),
//                leaving one bit per sample and 8-sample block sums;
//   marks warp   pre/post windows and merge (rows 3-4), the tile aggregate
//                (published for the look-back), Q partial bins (rows 7-8);
//   look-back    decoupled look-back over earlier tiles' published states
//                (two warps, alternate tiles): the tile's exclusive prefix
//                (pool row, island index, entering run);
//   loader       once a tile's prefix is known, bulk-copies the tile proper
//                (still in L2) into one of two input slots;
//   writers      stage the marked samples' rows at their global byte phase
//                (one of two stage buffers), store them with one bulk copy
//                plus unaligned ends, and write the tile's island records
//                (row 5).
//
// Nothing waits for a tile that was not ticketed earlier, and a ticket is only
// taken when its record slot is free, so every ticketed tile is counted and
// published without waiting: the look-backs always end.  Every wait is
// bounded (kWaitLimitNs), after which the CTA flags DAQ_DEV_TIMEOUT and stops.
#pragma once

#include "daq_steps.cuh"
#include "daq_twopass.cuh"

namespace daq {

constexpr int kStrProducer = 0;
constexpr int kStrCount0 = 1;
constexpr int kStrNCount = 12;
constexpr int kStrMarks = kStrCount0 + kStrNCount;
constexpr int kStrLook = kStrMarks + 1;
constexpr int kStrNLook = 2;
constexpr int kStrLoader = kStrLook + kStrNLook;
constexpr int kStrWriter0 = kStrLoader + 1;
constexpr int kStrNWriter = 8;
constexpr int kStrWarps = kStrWriter0 + kStrNWriter;
constexpr int kStrThreads = 32 * kStrWarps;
constexpr int kStrNMeta = 8;   // tiles in flight per CTA
constexpr int kStrNSlot = 2;   // compaction input slots (tile proper)
constexpr int kStrNStage = 2;  // row stages
constexpr int kStrStrip = 256; // samples per count-warp strip (8 per lane)
constexpr int kStrWriterBar = 1;  // named barrier of the writer warps

template <int TW> struct StreamMeta {
    TileInfo T;
    Agg agg, excl;
    uint8_t abyte[128];  // threshold bits of the extended tile (4 strips at most)
    int32_t blocksum[TW / 8];
    uint32_t wm[TW / 32], ws[TW / 32], we[TW / 32];
    int32_t wmb[TW / 32], wsb[TW / 32], wls[TW / 32];
};

enum {
    kSBarMetaFull = 0,
    kSBarBits = kSBarMetaFull + kStrNMeta,
    kSBarAgg = kSBarBits + kStrNMeta,
    kSBarExcl = kSBarAgg + kStrNMeta,
    kSBarMetaFree = kSBarExcl + kStrNMeta,
    kSBarSlotFull = kSBarMetaFree + kStrNMeta,
    kSBarSlotEmpty = kSBarSlotFull + kStrNSlot,
    kSNBars = kSBarSlotEmpty + kStrNSlot
};

template <int TW> __host__ __device__ constexpr size_t stream_meta_bytes()
{
    return (sizeof(StreamMeta<TW>) + 15) & ~size_t(15);
}

__host__ __device__ inline size_t stream_stage_bytes(int tw, int X) { return ((size_t)tw * 2 * X + 32 + 15) & ~size_t(15); }

// Shared-memory layout: slots, stages, tile records, sample sums (decimation
// factors that are not multiples of 8), barriers, fill plan, end marker.
template <int TW> struct StreamSmem {
    size_t slot0, stage0, meta0, sarr0, bars, fts, lens, end, total;
    __host__ __device__ StreamSmem(int X, int slot_bytes_b, int need_sarr)
    {
        slot0 = 0;
        stage0 = slot0 + (size_t)kStrNSlot * slot_bytes_b;
        meta0 = stage0 + (size_t)kStrNStage * stream_stage_bytes(TW, X);
        sarr0 = meta0 + (size_t)kStrNMeta * stream_meta_bytes<TW>();
        bars = (sarr0 + (need_sarr ? (size_t)kStrNMeta * TW * 4 : 0) + 15) & ~size_t(15);
        fts = bars + (size_t)kSNBars * 8;
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

// Warp-uniform form of stream_wait.
__device__ __forceinline__ int stream_wait_warp(const KArgs &a, uint64_t *bar, uint32_t parity, long long i,
                                                const volatile long long *s_end)
{
    int r = stream_wait(a, bar, parity, i, s_end);
    r = __shfl_sync(kFull, r, 0);  // lane 0 decides; the others' view of the phase is the same or later
    return r;
}

__device__ __forceinline__ uint4 ldg_v4_hint(const int16_t *p, uint64_t pol)
{
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

// One strip of the extended tile (one warp): extended columns [256 k, 256 k + 256),
// lane L owning columns 256 k + 8 L ... + 7.  Crystal words are loaded six
// crystals at a time, the next six in flight while the current six are added.
// Writes the strip's 32 bytes of threshold bits, its 8-sample block sums and
// (need_sarr) per-sample sums of the tile proper.
template <int TW>
__device__ __forceinline__ void stream_count_strip(const KArgs &a, const TileInfo &T, int k, uint8_t *abyte,
                                                   int32_t *blocksum, int32_t *sarr, uint64_t pol, int lane)
{
    constexpr int B = 6;
    const int X = a.n_xtal;
    const int cl = kStrStrip * k + 8 * lane;
    const long long t = T.t0 - a.hl + cl;
    const bool in_ext = cl < a.ew;
    // a group of 8 samples lies wholly inside or outside [0, n_samples): t and
    // n_samples are multiples of 8
    const bool ld_ok = in_ext && t >= 0 && t < a.n_samples;
    const long long pitch = a.n_samples;
    const int16_t *p = a.samples + ((long long)T.f * a.n_calo + T.c) * X * pitch + (ld_ok ? t : 0);
    int acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0;
    uint4 va[B], vb[B];
    auto issue = [&](uint4 *v, int x0) {
#pragma unroll
        for (int j = 0; j < B; ++j) {
            v[j] = make_uint4(0u, 0u, 0u, 0u);
            if (ld_ok && x0 + j < X) v[j] = ldg_v4_hint(p + (long long)(x0 + j) * pitch, pol);
        }
    };
    auto consume = [&](const uint4 *v) {
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const uint32_t w[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc[2 * q] = __dp2a_lo((int)w[q], 0x0001, acc[2 * q]);
                acc[2 * q + 1] = __dp2a_lo((int)w[q], 0x0100, acc[2 * q + 1]);
            }
        }
    };
    issue(va, 0);
    for (int x0 = 0; x0 < X; x0 += 2 * B) {
        issue(vb, x0 + B);
        consume(va);
        issue(va, x0 + 2 * B);
        consume(vb);
    }
    uint32_t bits = 0;
    int S[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        S[j] = acc[j] - T.ptot;
        const bool in = in_ext && t + j >= 0 && t + j < T.len;
        bits |= (uint32_t)(in && S[j] > a.threshold) << j;
    }
    abyte[32 * k + lane] = (uint8_t)bits;
    const int cp = cl - a.hl;  // column within the tile proper (a multiple of 8)
    if (in_ext && cp >= 0 && cp < TW) {
        int bs = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (t + j < T.t_end) bs += S[j];
        blocksum[cp >> 3] = bs;
        if (a.need_sarr) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (t + j < T.t_end) sarr[cp + j] = S[j];
        }
    }
}

template <int TW>
__global__ void __launch_bounds__(kStrThreads, 1) daq_stream_kernel(const __grid_constant__ KArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int X = a.n_xtal;
    const StreamSmem<TW> L(X, a.slot_bytes_b, a.need_sarr);
    const size_t stage_bytes = stream_stage_bytes(TW, X);
    constexpr size_t meta_bytes = stream_meta_bytes<TW>();
    unsigned char *slot0 = smem + L.slot0;
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
    const int n_strips = (a.ew + kStrStrip - 1) / kStrStrip;

    if (tid == 0) *s_end = 0x7fffffffffffffffll;
    const PlanView plan = cache_plan(a, fts_s, lens_s, tid, kStrThreads);
    for (int m = 0; m < kStrNMeta; ++m)
        for (int i = tid; i < 32; i += kStrThreads) reinterpret_cast<uint32_t *>(meta(m)->abyte)[i] = 0u;
    if (tid == 0) {
        for (int m = 0; m < kStrNMeta; ++m) {
            mbar_init(bars + kSBarMetaFull + m, 1);
            mbar_init(bars + kSBarBits + m, kStrNCount);
            mbar_init(bars + kSBarAgg + m, 1);
            mbar_init(bars + kSBarExcl + m, 1);
            mbar_init(bars + kSBarMetaFree + m, 1);
        }
        for (int s = 0; s < kStrNSlot; ++s) {
            mbar_init(bars + kSBarSlotFull + s, 1);
            mbar_init(bars + kSBarSlotEmpty + s, 1);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const long long total = plan.fts[a.n_fills];
    const bool skip_isl = (a.flags & DAQ_SKIP_ISLANDS) != 0;
    const bool skip_q = (a.flags & DAQ_SKIP_Q) != 0;

    if (warp == kStrProducer) {
        // ------------------------------------------------------------ tickets, decode, L2 prefetch
        if (lane == 0) {
            for (long long i = 0;; ++i) {
                const int m = (int)(i % kStrNMeta);
                if (i >= kStrNMeta &&
                    stream_wait(a, bars + kSBarMetaFree + m, (uint32_t)((i / kStrNMeta - 1) & 1), i, nullptr) != 1)
                    break;
                StreamMeta<TW> *M = meta(m);
                const long long tk = (long long)atomicAdd(a.ticket, 1u);
                if (!decode_tile<TW>(a, tk, M->T, plan.fts, plan.lens)) {
                    M->T.tile = -1;
                    *s_end = i;
                    mbar_arrive(bars + kSBarMetaFull + m);
                    break;
                }
                trace_stamp(a, tk, 0);
                trace_value(a, tk, 10, sm_id());
                trace_value(a, tk, 11, TW);
                issue_tile_prefetch(a, M->T);
                trace_stamp(a, tk, 1);
                mbar_arrive(bars + kSBarMetaFull + m);
            }
        }
    } else if (warp >= kStrCount0 && warp < kStrCount0 + kStrNCount) {
        // ------------------------------------------------------------ crystal sums, threshold bits
        // Every count warp passes every tile in order and arrives on its bits
        // barrier once (after its strips, if it has any), so no count warp is
        // ever more than one phase ahead of or behind a barrier it waits on.
        const int cw = warp - kStrCount0;
        const uint64_t pol = l2_policy_evict_last();
        for (long long i = 0;; ++i) {
            const int m = (int)(i % kStrNMeta);
            const int r = stream_wait_warp(a, bars + kSBarMetaFull + m, (uint32_t)((i / kStrNMeta) & 1), i, s_end);
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile >= 0) {
                // strips g = i * n_strips + k with g % kStrNCount == cw
                const long long g0 = i * n_strips;
                for (int k = (int)(((cw - g0) % kStrNCount + kStrNCount) % kStrNCount); k < n_strips;
                     k += kStrNCount) {
                    if (k == 0 && lane == 0) trace_stamp(a, T.tile, 2);
                    stream_count_strip<TW>(a, T, k, M->abyte, M->blocksum, sarr(m), pol, lane);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bars + kSBarBits + m);
            if (T.tile < 0) break;
        }
    } else if (warp == kStrMarks) {
        // ------------------------------------------------------------ windows, merge, aggregate, Q
        for (long long i = 0;; ++i) {
            const int m = (int)(i % kStrNMeta);
            const int r = stream_wait_warp(a, bars + kSBarBits + m, (uint32_t)((i / kStrNMeta) & 1), i, s_end);
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) {
                if (lane == 0) mbar_arrive(bars + kSBarAgg + m);
                break;
            }
            if (lane == 0) trace_stamp(a, T.tile, 3);
            const Agg agg = tile_bits<TW>(a, T, M->abyte, words(m), nullptr, lane);
            if (lane == 0) {
                M->agg = agg;
                if (T.tile > 0) publish(a.status, T.tile, false, agg);
                trace_stamp(a, T.tile, 4);
            }
            if (!skip_q) q_partial(a, T, M->blocksum, sarr(m), lane, 32);
            __syncwarp();
            if (lane == 0) mbar_arrive(bars + kSBarAgg + m);
        }
    } else if (warp >= kStrLook && warp < kStrLook + kStrNLook) {
        // ------------------------------------------------------------ decoupled look-back
        for (long long i = warp - kStrLook;; i += kStrNLook) {
            const int m = (int)(i % kStrNMeta);
            const int r = stream_wait_warp(a, bars + kSBarAgg + m, (uint32_t)((i / kStrNMeta) & 1), i, s_end);
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) {
                if (lane == 0) mbar_arrive(bars + kSBarExcl + m);
                break;
            }
            const Agg agg = M->agg;
            if (lane == 0) trace_stamp(a, T.tile, 5);
            unsigned lb_stats = 0;
            const Agg excl = T.tile > 0 ? look_back(a, T.tile, lane, &lb_stats) : agg_identity();
            if (lane == 0) {
                publish(a.status, T.tile, true, combine(excl, agg));
                M->excl = excl;
                trace_stamp(a, T.tile, 6);
                trace_value(a, T.tile, 14, lb_stats);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bars + kSBarExcl + m);
        }
    } else if (warp == kStrLoader) {
        // ------------------------------------------------------------ tile proper -> input slot (from L2)
        if (lane == 0) {
            const uint32_t box_bytes = (uint32_t)a.nbox_b * (uint32_t)X * (uint32_t)a.rs_b;
            uint32_t pending = 0, pend_par = 0;  // per slot: a load issued and its phase parity
            for (long long i = 0;; ++i) {
                const int m = (int)(i % kStrNMeta), s = (int)(i % kStrNSlot);
                if (stream_wait(a, bars + kSBarExcl + m, (uint32_t)((i / kStrNMeta) & 1), i, s_end) != 1) break;
                if (i >= kStrNSlot &&
                    stream_wait(a, bars + kSBarSlotEmpty + s, (uint32_t)((i / kStrNSlot - 1) & 1), i, nullptr) != 1)
                    break;
                pending &= ~(1u << s);
                StreamMeta<TW> *M = meta(m);
                const TileInfo T = M->T;
                if (T.tile < 0) {
                    mbar_arrive(bars + kSBarSlotFull + s);
                    break;
                }
                if (skip_isl || M->agg.m == 0 || M->excl.poison) {
                    mbar_arrive(bars + kSBarSlotFull + s);  // nothing to stage
                } else {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(bars + kSBarSlotFull + s, box_bytes);
                    issue_tile_load_b(a, T, slot0 + (size_t)s * a.slot_bytes_b, bars + kSBarSlotFull + s);
                    pending |= 1u << s;
                    pend_par = (pend_par & ~(1u << s)) | ((uint32_t)((i / kStrNSlot) & 1) << s);
                    trace_stamp(a, T.tile, 12);
                }
            }
            // copies still in flight land before this CTA may exit
            for (int s = 0; s < kStrNSlot; ++s)
                if (pending & (1u << s)) mbar_wait_bounded(bars + kSBarSlotFull + s, (pend_par >> s) & 1u, kWaitLimitNs);
        }
    } else {
        // ------------------------------------------------------------ writers
        const int wt = tid - 32 * kStrWriter0, ww = warp - kStrWriter0;
        constexpr int nthr = 32 * kStrNWriter;
        const long long rb = 2ll * X;
        int last_use[kStrNStage];  // bulk groups committed since each stage's last group (-1: none pending)
        for (int o = 0; o < kStrNStage; ++o) last_use[o] = -1;
        bool any_store = false;
        for (long long i = 0;; ++i) {
            const int m = (int)(i % kStrNMeta), s = (int)(i % kStrNSlot), o = (int)(i % kStrNStage);
            int r = 0;
            if (ww == 0) r = stream_wait_warp(a, bars + kSBarSlotFull + s, (uint32_t)((i / kStrNSlot) & 1), i, s_end);
            r = __shfl_sync(kFull, r, 0);
            // all writer warps learn the outcome through shared memory
            __shared__ int s_r;
            if (wt == 0) s_r = r;
            asm volatile("bar.sync %0, %1;" ::"n"(kStrWriterBar), "n"(nthr) : "memory");
            r = s_r;
            if (r != 1) break;
            StreamMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) break;
            const Agg agg = M->agg, excl = M->excl;
            if (wt == 0) trace_stamp(a, T.tile, 8);
            const bool rows = !skip_isl && agg.m > 0 && !excl.poison;
            unsigned char *stage = stage0 + (size_t)o * stage_bytes;
            const long long gs = excl.m * rb;
            const int phase = (int)(gs & 15);
            if (rows) {
                if (wt == 0) {
                    // the stage is free once its last bulk store has read it
                    if (last_use[o] == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    else if (last_use[o] == 1) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    last_use[o] = -1;
                    trace_stamp(a, T.tile, 13);
                }
                asm volatile("bar.sync %0, %1;" ::"n"(kStrWriterBar), "n"(nthr) : "memory");
                const int nt = (int)(T.t_end - T.t0);
                const TileWords W = words(m);
                const uint32_t slot_s = smem_addr(slot0 + (size_t)s * a.slot_bytes_b);
                for (int it = ww; it < (nt + 63) / 64; it += kStrNWriter)
                    compact_step(a, slot_s, it, nt, W.m, W.mb, stage, phase, lane);
            }
            asm volatile("bar.sync %0, %1;" ::"n"(kStrWriterBar), "n"(nthr) : "memory");
            if (wt == 0) {
                mbar_arrive(bars + kSBarSlotEmpty + s);
                trace_stamp(a, T.tile, 7);
            }
            if (rows) {
                long long ge = gs + agg.m * rb;
                const long long cap_b = a.pool_cap * rb;
                if (ge > cap_b) {
                    ge = cap_b;
                    if (wt == 0) set_status_bit(a, DAQ_DEV_POOL_OVERFLOW);
                }
                if (ge > gs) {
                    unsigned char *g = reinterpret_cast<unsigned char *>(a.pool);
                    long long a16 = (gs + 15) & ~15ll, b16 = ge & ~15ll;
                    if (a16 > ge) a16 = ge;
                    if (b16 < a16) b16 = a16;
                    if (wt == 0 && b16 > a16) {
                        fence_proxy_async_smem();
                        bulk_s2g_hint(g + a16, stage + phase + (a16 - gs), (uint32_t)(b16 - a16),
                                      l2_policy_evict_first());
                        bulk_commit();
                        for (int q = 0; q < kStrNStage; ++q)
                            if (last_use[q] >= 0) ++last_use[q];
                        last_use[o] = 0;
                        any_store = true;
                    }
                    const int n_head = (int)((a16 - gs) >> 1), n_tail = (int)((ge - b16) >> 1);
                    if (wt >= 64 && wt < 64 + n_head)
                        *reinterpret_cast<uint16_t *>(g + gs + 2 * (wt - 64)) =
                            *reinterpret_cast<const uint16_t *>(stage + phase + 2 * (wt - 64));
                    else if (wt >= 96 && wt < 96 + n_tail) {
                        const long long off = b16 + 2 * (wt - 96);
                        *reinterpret_cast<uint16_t *>(g + off) =
                            *reinterpret_cast<const uint16_t *>(stage + phase + (off - gs));
                    }
                }
                if (ww == 0) write_headers<TW>(a, T, words(m), excl, lane);
            }
            if (ww == 0) {
                if (lane == 0 && T.tile == total - 1) write_counts(a, T.tile, combine(excl, agg));
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(bars + kSBarMetaFree + m);
                    trace_stamp(a, T.tile, 9);
                }
            }
        }
        if (wt == 0 && any_store) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

}  // namespace daq
