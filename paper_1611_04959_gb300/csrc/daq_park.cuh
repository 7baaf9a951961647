// Single-read form (daq_params.grid = -6): every sample is read from HBM once,
// and a tile's rows wait for their place in the pool in Tensor Memory.
//
// A tile's pool rows can only be written once its exclusive prefix (the pool
// rows of all earlier tiles) is known, several microseconds of cross-CTA
// look-back after the tile has been read.  Shared memory cannot hold the tiles
// waiting that long at full rate beside the tiles being loaded.  The SM's
// Tensor Memory (256 KB, otherwise unused: nothing on this path is a matrix
// product) can.  The crystal-sum loop already holds, in registers, the row
// words of the samples it sums (two crystals of one sample per 32-bit word), so
// it writes them straight into Tensor Memory; once the prefix is known they are
// read back, the marked rows are staged in shared memory at their global byte
// phase and written with one bulk copy, as in the two-pass compaction.
//
// One persistent CTA per SM; warps have fixed roles and hand tiles to each
// other through mbarriers over a ring of tile records:
//
//   producer     takes a ticket (tiles run in ticket order), decodes the tile
//                and bulk-copies its crystal rows plus halo into one of two
//                count slots (2-D tensor boxes);
//   sum warps    crystal sums (Table 2 row 6) minus the summed pedestals
//                (row 1), threshold bits (row 2), 8-sample block sums, and the
//                raw rows of the samples into a park slot of Tensor Memory;
//   marks warps  pre/post windows and merge (rows 3-4), the tile aggregate
//                (published for the look-back), Q partial bins (rows 7-8);
//                two warps take alternate tiles;
//   look-back    decoupled look-back over earlier tiles' published states
//                (four warps, tiles in turn): the tile's exclusive prefix;
//   stage warps  (two per Tensor Memory lane quadrant, taking its steps in
//                turn) once the prefix is known, read the rows back and store
//                the marked ones at phase + rank * 2 n_xtal bytes of an
//                out-stage, rank = the sample's pool row within the tile from
//                the marks words (row 5);
//   bulk warp    one bulk copy of the out-stage to the pool (plus unaligned
//                ends);
//   record warp  the tile's island records and, after the last tile, the
//                call's counts.
//
// Park slot layout: step it (extended columns 64 it + 2 l and + 1 for lane l)
// is summed by sum warp w = 1 + it % 8, which writes lane 32 (w % 4) + l of
// cps columns from col(it): column col + 2 k holds word k (crystals 2k, 2k + 1)
// of the row of extended column 64 it + 2 l, column col + 2 k + 1 that of
// column 64 it + 2 l + 1.  The two sum warps of one quadrant take alternate
// column blocks.
//
// As in the streaming form, nothing waits for a tile ticketed later, and a
// ticket is only taken when a record and a count slot are free, so every
// ticketed tile is counted and published: a tile's aggregate needs only its own
// load, sums and marks.  Everything else a tile waits for (a park slot, an
// out-stage) is held by tiles ticketed before it.  Every wait is bounded; a
// CTA that gives up flags DAQ_DEV_TIMEOUT, which makes the other CTAs stop
// too.  Every exit path goes through one final barrier, after which the
// allocating warp frees the Tensor Memory.
#pragma once

#include "daq_steps.cuh"
#include "daq_stream.cuh"
#include "daq_twopass.cuh"

namespace daq {

constexpr int kPkProducer = 0;
constexpr int kPkSum0 = 1;
constexpr int kPkNSum = 8;
constexpr int kPkMarks = kPkSum0 + kPkNSum;
constexpr int kPkNMarks = 2;
constexpr int kPkLook = kPkMarks + kPkNMarks;
constexpr int kPkNLook = 4;
constexpr int kPkRec = kPkLook + kPkNLook;
constexpr int kPkStage0 = kPkRec + 1;
constexpr int kPkNStage = 8;  // two per Tensor Memory quadrant
constexpr int kPkBulk = kPkStage0 + kPkNStage;
constexpr int kPkWarps = kPkBulk + 1;
constexpr int kPkThreads = 32 * kPkWarps;
constexpr int kPkNCSlot = 2;     // count slots (extended tile)
constexpr int kPkMaxOut = 2;     // out-stages (1 or 2)
constexpr int kPkMaxMeta = 8;    // tile records per CTA (a multiple of 4)
constexpr int kPkMaxPark = 8;    // park slots
constexpr int kPkCols = 512;     // Tensor Memory columns taken (all of them)
static_assert(kPkStage0 % 4 == 0, "quadrant q of Tensor Memory is reached by warps with warp % 4 == q");
static_assert(kPkNSum == 8, "two sum warps per Tensor Memory quadrant");

template <int TW> struct ParkMeta {
    TileInfo T;
    Agg agg, excl;
    uint8_t abyte[128];  // threshold bits of the extended tile
    int32_t blocksum[TW / 8];
    uint32_t wm[TW / 32], ws[TW / 32], we[TW / 32];
    int32_t wmb[TW / 32], wsb[TW / 32], wls[TW / 32];
};

template <int TW> __host__ __device__ constexpr size_t park_meta_bytes() { return (sizeof(ParkMeta<TW>) + 15) & ~size_t(15); }

// Out-stage: a tile's marked rows (2 n_xtal bytes each) after a byte phase < 16.
__host__ __device__ inline size_t park_out_bytes(int tw, int X) { return ((size_t)tw * 2 * X + 16 + 127) & ~size_t(127); }

// Tensor Memory columns of one step's rows (two rows of n_xtal / 2 words,
// interleaved), in whole 16-column loads.
__host__ __device__ inline int park_step_cols(int X) { return (X + 15) / 16 * 16; }

// Columns of one park slot: the steps of one quadrant (two per round of eight
// steps).
__host__ __device__ inline int park_slot_cols(int ew, int X) { return 2 * ((ew + 511) / 512) * park_step_cols(X); }

// Column (within a park slot) of step it's rows, in the quadrant of its sum warp.
__host__ __device__ inline int park_step_col(int it, int cps) { return (2 * (it / kPkNSum) + (it % kPkNSum) / 4) * cps; }

// mbarrier indices
struct ParkBars {
    int nm, no, np;
    __host__ __device__ int bits(int m) const { return m; }
    __host__ __device__ int agg(int m) const { return nm + m; }
    __host__ __device__ int excl(int m) const { return 2 * nm + m; }
    __host__ __device__ int meta_free(int m) const { return 3 * nm + m; }
    __host__ __device__ int cfull(int s) const { return 4 * nm + s; }
    __host__ __device__ int cempty(int s) const { return 4 * nm + kPkNCSlot + s; }
    __host__ __device__ int ofull(int o) const { return 4 * nm + 2 * kPkNCSlot + o; }
    __host__ __device__ int ofree(int o) const { return 4 * nm + 2 * kPkNCSlot + no + o; }
    __host__ __device__ int pfull(int p) const { return 4 * nm + 2 * kPkNCSlot + 2 * no + p; }
    __host__ __device__ int pfree(int p) const { return 4 * nm + 2 * kPkNCSlot + 2 * no + np + p; }
    __host__ __device__ int count() const { return 4 * nm + 2 * kPkNCSlot + 2 * no + 2 * np; }
};
// arrivals that free a tile record: the marks warp (after its Q bins), the
// stage warps, the bulk warp and the record warp
constexpr int kPkMetaFreeArrivals = 1 + kPkNStage + 1 + 1;

// Shared-memory layout: count slots, out-stages, tile records, sample sums
// (decimation factors that are not multiples of 8), barriers, fill plan, end
// marker and Tensor Memory address.
template <int TW> struct ParkSmem {
    size_t cslot0, out0, meta0, sarr0, bars, fts, lens, misc, total;
    __host__ __device__ ParkSmem(int X, int slot_bytes, int need_sarr, int nm, int no, int np)
    {
        cslot0 = 0;
        out0 = cslot0 + (size_t)kPkNCSlot * slot_bytes;
        meta0 = out0 + (size_t)no * park_out_bytes(TW, X);
        sarr0 = meta0 + (size_t)nm * park_meta_bytes<TW>();
        bars = (sarr0 + (need_sarr ? (size_t)nm * TW * 4 : 0) + 15) & ~size_t(15);
        fts = bars + (size_t)ParkBars{nm, no, np}.count() * 8;
        lens = fts + 8 * (size_t)(kPlanSmem + 1);
        misc = (lens + 4 * (size_t)kPlanSmem + 15) & ~size_t(15);  // end marker (8 B), Tensor Memory address (4 B)
        total = (misc + 16 + 127) & ~size_t(127);
    }
};

// Bounded mbarrier wait without a suspend-time hint (tile handoffs are short),
// one thread: 1 when the phase completed, 0 when the stream ended before use i
// (*s_end < i), -1 on timeout or once another CTA has flagged one.
__device__ __forceinline__ int park_wait1(const KArgs &a, uint64_t *bar, uint32_t parity, long long i,
                                          const volatile long long *s_end)
{
    if (mbar_try_wait(bar, parity)) return 1;
    const uint64_t t0 = global_ns();
    for (uint32_t k = 1;; ++k) {
        if (mbar_try_wait(bar, parity)) return 1;
        if (s_end && *s_end < i) return 0;
        if ((k & 63u) == 0u) {
            if (global_ns() - t0 > kWaitLimitNs) {
                set_status_bit(a, DAQ_DEV_TIMEOUT);
                return -1;
            }
            if (aborted(a)) return -1;
        }
    }
}

// park_wait1 by a whole warp (lane 0's outcome).
__device__ __forceinline__ int park_wait(const KArgs &a, uint64_t *bar, uint32_t parity, long long i,
                                         const volatile long long *s_end)
{
    const int r = park_wait1(a, bar, parity, i, s_end);
    return __shfl_sync(kFull, r, 0);
}

__device__ __forceinline__ void sts_u32(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// One warp step of the crystal sum (as sum_pass_step: lane L owns extended
// columns c = 64 it + 2L, c + 1) that also writes the two samples' raw rows to
// Tensor Memory at column tcol of the warp's quadrant (see the layout above):
// sixteen row words (eight crystal pairs) per tcgen05.st.  n_xtal is even.
// Every lane runs the crystal loop (the stores are warp-wide); lanes past the
// extended tile sum zeros.
__device__ __forceinline__ void park_sum_step(const KArgs &a, const TileInfo &T, uint32_t slot_s, int it, int nbt,
                                              uint8_t *abyte, int32_t *blocksum, int32_t *sarr, uint32_t tcol,
                                              bool rows, int lane)
{
    const int X = a.n_xtal;
    const int c = 64 * it + 2 * lane;
    const bool have = c < a.ew;  // ew is even, so c + 1 < ew too
    const int k = (c >= a.boxw) + (c >= 2 * a.boxw) + (c >= 3 * a.boxw) + (c >= 4 * a.boxw);
    const uint32_t base = slot_s + (uint32_t)(k * a.box_stride + 2 * (c - k * a.boxw));
    const long long t = T.t0 - a.hl + c;
    int acc0 = 0, acc1 = 0, acc0b = 0, acc1b = 0;
    for (int x0 = 0; x0 < X; x0 += 16) {
        uint32_t v[16];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int x = x0 + 2 * u;
            uint32_t w0 = 0u, w1 = 0u;
            if (have && x < X) {
                w0 = lds_u32(base + (uint32_t)(x * a.rs));
                w1 = lds_u32(base + (uint32_t)((x + 1) * a.rs));
            }
            acc0 = __dp2a_lo((int)w0, 0x0001, acc0);
            acc1 = __dp2a_lo((int)w0, 0x0100, acc1);
            acc0b = __dp2a_lo((int)w1, 0x0001, acc0b);
            acc1b = __dp2a_lo((int)w1, 0x0100, acc1b);
            v[2 * u] = __byte_perm(w0, w1, 0x5410);
            v[2 * u + 1] = __byte_perm(w0, w1, 0x7632);
        }
        if (rows) tmem_st16(tcol + (uint32_t)x0, v);
    }
    acc0 += acc0b;
    acc1 += acc1b;
    const int S0 = acc0 - T.ptot, S1 = acc1 - T.ptot;
    const bool in0 = have && t >= 0 && t < T.len, in1 = have && t + 1 >= 0 && t + 1 < T.len;
    const uint32_t be = __ballot_sync(kFull, in0 && S0 > a.threshold);
    const uint32_t bo = __ballot_sync(kFull, in1 && S1 > a.threshold);
    if (lane == 0) {
        const unsigned long long m = spread_bits(be) | (spread_bits(bo) << 1);
        *reinterpret_cast<uint2 *>(abyte + 8 * it) = make_uint2((uint32_t)m, (uint32_t)(m >> 32));
    }
    const int cp = c - a.hl;  // column within the tile proper
    const bool proper = have && cp >= 0 && cp < 8 * nbt;
    int sv = (proper && t < T.t_end ? S0 : 0) + (proper && t + 1 < T.t_end ? S1 : 0);
    sv += __shfl_xor_sync(kFull, sv, 1);
    sv += __shfl_xor_sync(kFull, sv, 2);
    if (proper && (lane & 3) == 0) blocksum[cp >> 3] = sv;
    if (a.need_sarr && proper) {
        if (t < T.t_end) sarr[cp] = S0;
        if (t + 1 < T.t_end) sarr[cp + 1] = S1;
    }
}

template <int TW>
__global__ void __launch_bounds__(kPkThreads, 1) daq_park_kernel(const __grid_constant__ KArgs a)
{
    constexpr int NBT = TW / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int X = a.n_xtal;
    const int NM = a.str_meta, NO = a.str_stages, NP = a.pk_slots, PC = a.pk_cols;
    const int cps = park_step_cols(X);
    const ParkBars BI{NM, NO, NP};
    const ParkSmem<TW> L(X, a.slot_bytes, a.need_sarr, NM, NO, NP);
    const size_t out_bytes = park_out_bytes(TW, X);
    constexpr size_t meta_bytes = park_meta_bytes<TW>();
    unsigned char *cslot0 = smem + L.cslot0;
    unsigned char *out0 = smem + L.out0;
    unsigned char *meta0 = smem + L.meta0;
    int32_t *sarr0 = reinterpret_cast<int32_t *>(smem + L.sarr0);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    long long *fts_s = reinterpret_cast<long long *>(smem + L.fts);
    int32_t *lens_s = reinterpret_cast<int32_t *>(smem + L.lens);
    volatile long long *s_end = reinterpret_cast<volatile long long *>(smem + L.misc);
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(smem + L.misc + 8);
    auto meta = [&](int m) { return reinterpret_cast<ParkMeta<TW> *>(meta0 + (size_t)m * meta_bytes); };
    auto sarr = [&](int m) { return sarr0 + (a.need_sarr ? m * TW : 0); };
    auto words = [&](int m) {
        ParkMeta<TW> *M = meta(m);
        return TileWords{M->wm, M->ws, M->we, M->wmb, M->wsb, M->wls};
    };
    auto bar = [&](int idx) { return bars + idx; };
    auto par = [](long long i, int n) { return (uint32_t)((i / n) & 1); };           // phase of use i of a ring of n
    auto par_prev = [](long long i, int n) { return (uint32_t)((i / n - 1) & 1); };  // phase of use i - n

    // Tensor Memory: this CTA is the only one on its SM (one CTA per SM by its
    // registers and shared memory), so the allocation is granted at once.
    if (warp == kPkStage0) {
        tmem_alloc(s_taddr, kPkCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        *s_end = 0x7fffffffffffffffll;
        for (int m = 0; m < NM; ++m) {
            mbar_init(bar(BI.bits(m)), kPkNSum);
            mbar_init(bar(BI.agg(m)), 1);
            mbar_init(bar(BI.excl(m)), 1);
            mbar_init(bar(BI.meta_free(m)), kPkMetaFreeArrivals);
        }
        for (int s = 0; s < kPkNCSlot; ++s) {
            mbar_init(bar(BI.cfull(s)), 1);
            mbar_init(bar(BI.cempty(s)), kPkNSum);
        }
        for (int o = 0; o < NO; ++o) {
            mbar_init(bar(BI.ofull(o)), kPkNStage);
            mbar_init(bar(BI.ofree(o)), 1);
        }
        for (int p = 0; p < NP; ++p) {
            mbar_init(bar(BI.pfull(p)), kPkNSum);
            mbar_init(bar(BI.pfree(p)), kPkNStage);
        }
        fence_mbar_init();
    }
    for (int m = 0; m < NM; ++m)
        for (int i = tid; i < 32; i += kPkThreads) reinterpret_cast<uint32_t *>(meta(m)->abyte)[i] = 0u;
    pdl_wait();  // the prepare kernel's plan, pedestals and resets
    const PlanView plan = cache_plan(a, fts_s, lens_s, tid, kPkThreads);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tbase = *s_taddr;

    const long long total = plan.fts[a.n_fills];
    const bool skip_isl = (a.flags & DAQ_SKIP_ISLANDS) != 0;
    const bool skip_q = (a.flags & DAQ_SKIP_Q) != 0;
    const int wpr = a.wpr;  // 32-bit words per pool row (n_xtal even)
    const long long rb = 2ll * X;
    const int n_steps = (a.ew + 63) / 64;

    if (warp == kPkProducer) {
        // ------------------------------------------------------------ tickets, decode, count-slot loads
        if (lane == 0) {
            uint32_t pending = 0, pend_par = 0;  // per count slot: a load issued, its phase parity
            for (long long i = 0;; ++i) {
                const int m = (int)(i % NM), s = (int)(i % kPkNCSlot);
                if (i >= NM && park_wait1(a, bar(BI.meta_free(m)), par_prev(i, NM), i, nullptr) != 1) break;
                if (i >= kPkNCSlot && park_wait1(a, bar(BI.cempty(s)), par_prev(i, kPkNCSlot), i, nullptr) != 1)
                    break;
                ParkMeta<TW> *M = meta(m);
                const long long tk = aborted(a) ? total : (long long)atomicAdd(a.ticket, 1u);
                if (!decode_tile<TW>(a, tk, M->T, plan.fts, plan.lens)) {
                    M->T.tile = -1;
                    *s_end = i;
                    // the slot's last load has been consumed (cempty above), and
                    // this arrival completes one more phase of its barrier
                    pending &= ~(1u << s);
                    mbar_arrive(bar(BI.cfull(s)));
                    break;
                }
                trace_stamp(a, tk, 0);
                trace_value(a, tk, 10, sm_id());
                trace_value(a, tk, 11, TW);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar(BI.cfull(s)), tile_load_bytes(a));
                issue_tile_load(a, M->T, cslot0 + (size_t)s * a.slot_bytes, bar(BI.cfull(s)));
                pending |= 1u << s;
                pend_par = (pend_par & ~(1u << s)) | (par(i, kPkNCSlot) << s);
                trace_stamp(a, tk, 1);
            }
            // bulk copies still in flight land before this CTA may exit
            for (int s = 0; s < kPkNCSlot; ++s)
                if (pending & (1u << s)) mbar_wait_bounded(bar(BI.cfull(s)), (pend_par >> s) & 1u, kWaitLimitNs);
        }
    } else if (warp >= kPkSum0 && warp < kPkSum0 + kPkNSum) {
        // ------------------------------------------------------------ crystal sums, threshold bits, rows -> Tensor Memory
        const int sw = warp - kPkSum0;
        const uint32_t tq = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
        for (long long i = 0;; ++i) {
            const int m = (int)(i % NM), s = (int)(i % kPkNCSlot), p = (int)(i % NP);
            int r = park_wait(a, bar(BI.cfull(s)), par(i, kPkNCSlot), i, s_end);
            if (r == 1 && i >= NP) r = park_wait(a, bar(BI.pfree(p)), par_prev(i, NP), i, nullptr);
            if (r != 1) break;
            ParkMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile >= 0) {
                tmem_fence_after_sync();  // the park slot's previous rows have been read back
                if (sw == 0 && lane == 0) trace_stamp(a, T.tile, 2);
                const uint32_t slot_s = smem_addr(cslot0 + (size_t)s * a.slot_bytes);
                for (int it = sw; it < n_steps; it += kPkNSum)
                    park_sum_step(a, T, slot_s, it, NBT, M->abyte, M->blocksum, sarr(m),
                                  tq + (uint32_t)(p * PC + park_step_col(it, cps)), !skip_isl, lane);
                tmem_wait_st();
                tmem_fence_before_sync();
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar(BI.bits(m)));
                mbar_arrive(bar(BI.cempty(s)));
                mbar_arrive(bar(BI.pfull(p)));
            }
            if (T.tile < 0) break;
        }
    } else if (warp >= kPkMarks && warp < kPkMarks + kPkNMarks) {
        // ------------------------------------------------------------ windows, merge, aggregate, ranks, Q
        for (long long i = warp - kPkMarks;; i += kPkNMarks) {
            const int m = (int)(i % NM);
            const int r = park_wait(a, bar(BI.bits(m)), par(i, NM), i, s_end);
            if (r != 1) break;
            ParkMeta<TW> *M = meta(m);
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
            }
            __syncwarp();
            if (lane == 0) {
                trace_stamp(a, T.tile, 4);
                mbar_arrive(bar(BI.agg(m)));
            }
            if (!skip_q) q_partial(a, T, M->blocksum, sarr(m), lane, 32);
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(BI.meta_free(m)));
        }
    } else if (warp >= kPkLook && warp < kPkLook + kPkNLook) {
        // ------------------------------------------------------------ decoupled look-back (tiles in turn)
        for (long long i = warp - kPkLook;; i += kPkNLook) {
            const int m = (int)(i % NM);
            const int r = park_wait(a, bar(BI.agg(m)), par(i, NM), i, s_end);
            if (r != 1) break;
            ParkMeta<TW> *M = meta(m);
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
    } else if (warp == kPkRec) {
        // ------------------------------------------------------------ island records, counts
        for (long long i = 0;; ++i) {
            const int m = (int)(i % NM);
            const int r = park_wait(a, bar(BI.excl(m)), par(i, NM), i, s_end);
            if (r != 1) break;
            ParkMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) break;
            const Agg agg = M->agg, excl = M->excl;
            if (!skip_isl && agg.m > 0 && !excl.poison) write_headers<TW>(a, T, words(m), excl, lane);
            if (lane == 0 && T.tile == total - 1 && !excl.poison) write_counts(a, T.tile, combine(excl, agg));
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(BI.meta_free(m)));
        }
    } else if (warp >= kPkStage0 && warp < kPkStage0 + kPkNStage) {
        // ------------------------------------------------------------ Tensor Memory -> out-stage (marked rows)
        // Warps q and q + 4 share quadrant q and take its steps in turn.
        const int q = (warp - kPkStage0) & 3, half = (warp - kPkStage0) >> 2;
        const uint32_t tq = tbase + ((uint32_t)(32 * q) << 16);
        for (long long i = 0;; ++i) {
            const int m = (int)(i % NM), p = (int)(i % NP), o = (int)(i % NO);
            int r = park_wait(a, bar(BI.excl(m)), par(i, NM), i, s_end);
            ParkMeta<TW> *M = meta(m);
            if (r == 1 && M->T.tile < 0) break;
            if (r == 1) r = park_wait(a, bar(BI.pfull(p)), par(i, NP), i, nullptr);
            if (r == 1 && i >= NO) r = park_wait(a, bar(BI.ofree(o)), par_prev(i, NO), i, nullptr);
            if (r != 1) break;
            tmem_fence_after_sync();
            const TileInfo T = M->T;
            const Agg agg = M->agg, excl = M->excl;
            bool rows = !skip_isl && !excl.poison && agg.m > 0;
            if (rows && (a.flags & DAQ_DEBUG_CHECKS) && (excl.m < 0 || agg.m > T.t_end - T.t0)) {
                if (q == 0 && lane == 0) set_status_bit(a, DAQ_DEV_BAD_INDEX);  // more rows than the out-stage holds
                rows = false;
            }
            if (q == 0 && lane == 0) trace_stamp(a, T.tile, 8);
            if (rows) {
                const int nt = (int)(T.t_end - T.t0);
                const uint32_t out_s = smem_addr(out0 + (size_t)o * out_bytes) + (uint32_t)((excl.m * rb) & 15);
                // pool row within the tile of tile column c, -1 if unmarked (c, c + 1 share a marks word)
                const int ca0 = 2 * lane - a.hl;
                int nq = 0;  // steps of this quadrant so far
                for (int it = 0; it < n_steps; ++it) {
                    if (((kPkSum0 + it % kPkNSum) & 3) != q) continue;  // another quadrant's step
                    if ((nq++ & 1) != half) continue;                    // the other warp of the quadrant's
                    const int ca = 64 * it + ca0;                        // tile column of the lane's first sample
                    int ra = -1, rbk = -1;
                    if (ca >= 0 && ca < nt) {
                        const int w = ca >> 5, b = ca & 31;  // b even: ca + 1 is in the same word
                        const uint32_t mw = M->wm[w];
                        const int before = M->wmb[w] + __popc(mw & ((1u << b) - 1u));
                        if ((mw >> b) & 1u) ra = before;
                        if (ca + 1 < nt && ((mw >> (b + 1)) & 1u)) rbk = before + (int)((mw >> b) & 1u);
                    }
                    const uint32_t tcol = tq + (uint32_t)(p * PC + park_step_col(it, cps));
                    for (int x0 = 0; x0 < X; x0 += 16) {
                        uint32_t v[16];
                        tmem_ld16(tcol + (uint32_t)x0, v);
                        tmem_wait_ld();
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int kw = (x0 >> 1) + u;  // word of the row
                            if (kw < wpr) {
                                if (ra >= 0) sts_u32(out_s + 4u * (uint32_t)(ra * wpr + kw), v[2 * u]);
                                if (rbk >= 0) sts_u32(out_s + 4u * (uint32_t)(rbk * wpr + kw), v[2 * u + 1]);
                            }
                        }
                    }
                }
                fence_proxy_async_smem();  // the bulk copy reads the stage through the async proxy
            }
            tmem_fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar(BI.pfree(p)));
                mbar_arrive(bar(BI.ofull(o)));
                mbar_arrive(bar(BI.meta_free(m)));
            }
        }
    } else {
        // ------------------------------------------------------------ out-stage -> pool (bulk copy)
        // With two out-stages the copy of tile i is waited for (its reads of
        // the stage) once the copy of tile i + 1 has been issued; then the stage
        // and the tile record are released.
        unsigned char *gp = reinterpret_cast<unsigned char *>(a.pool);
        const long long cap_b = a.pool_cap * rb;
        long long prev = -1;  // iteration whose stage and record wait for their copy's reads
        for (long long i = 0;; ++i) {
            const int m = (int)(i % NM), o = (int)(i % NO);
            int r = park_wait(a, bar(BI.excl(m)), par(i, NM), i, s_end);
            ParkMeta<TW> *M = meta(m);
            if (r == 1 && M->T.tile < 0) break;
            if (r == 1) r = park_wait(a, bar(BI.ofull(o)), par(i, NO), i, nullptr);
            if (r != 1) break;
            const TileInfo T = M->T;
            const Agg agg = M->agg, excl = M->excl;
            unsigned char *stage = out0 + (size_t)o * out_bytes;
            const long long gs = excl.m * rb;
            const int phase = (int)(gs & 15);
            long long ge = gs + agg.m * rb;
            if (ge > cap_b) {
                ge = cap_b;
                if (lane == 0 && !skip_isl && !excl.poison) set_status_bit(a, DAQ_DEV_POOL_OVERFLOW);
            }
            const bool bad = (a.flags & DAQ_DEBUG_CHECKS) && (excl.m < 0 || agg.m > T.t_end - T.t0);
            if (!skip_isl && !excl.poison && !bad && ge > gs) {
                long long a16 = (gs + 15) & ~15ll, b16 = ge & ~15ll;
                if (a16 > ge) a16 = ge;
                if (b16 < a16) b16 = a16;
                if (lane == 0 && b16 > a16) {
                    fence_proxy_async_smem();
                    bulk_s2g(gp + a16, stage + phase + (a16 - gs), (uint32_t)(b16 - a16));
                }
                const int n_head = (int)((a16 - gs) >> 1), n_tail = (int)((ge - b16) >> 1);
                if (lane < n_head)
                    *reinterpret_cast<uint16_t *>(gp + gs + 2 * lane) =
                        *reinterpret_cast<const uint16_t *>(stage + phase + 2 * lane);
                else if (lane >= 16 && lane < 16 + n_tail) {
                    const long long off = b16 + 2 * (lane - 16);
                    *reinterpret_cast<uint16_t *>(gp + off) = *reinterpret_cast<const uint16_t *>(stage + phase + (off - gs));
                }
            }
            if (lane == 0) {
                bulk_commit();
                if (T.tile >= 0) trace_stamp(a, T.tile, 9);
                // with two stages the previous tile's copy has read its stage;
                // with one, this tile's copy
                if (NO > 1) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                else asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            }
            __syncwarp();
            const long long done = NO > 1 ? prev : i;
            if (done >= 0 && lane == 0) {
                mbar_arrive(bar(BI.ofree((int)(done % NO))));
                mbar_arrive(bar(BI.meta_free((int)(done % NM))));
            }
            prev = i;
        }
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }

    // every role is done; the Tensor Memory is freed by the warp that took it
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == kPkStage0) {
        tmem_fence_after_sync();
        tmem_dealloc(tbase, kPkCols);
    }
}

}  // namespace daq
