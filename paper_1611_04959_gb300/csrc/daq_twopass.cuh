// Two-pass form of the per-fill processing (the default path).
//
//   daq_count_kernel    every tile once, with its halo: crystal sums, pedestal
//                       subtraction, threshold, pre/post windows (the marks of
//                       the tile), Q-method partial bins; stores the tile's marks
//                       words and its aggregate (marked samples, island starts,
//                       trailing run).  No tile waits on another.
//   daq_scan_*_kernels  reduce-then-scan of the per-tile aggregates: every tile's
//                       exclusive prefix (pool row and island index it starts
//                       at, marked run entering it) and the call's totals.
//   daq_compact_kernel  every tile again (tile proper only): the raw samples of
//                       its marked times are transposed into rows in shared
//                       memory at the phase of their global position, written
//                       with one bulk copy (plus unaligned ends), and the tile's
//                       island records are written.
#pragma once

#include "daq_steps.cuh"

namespace daq {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;  // tiles per scan thread
constexpr int kScanChunk = kScanThreads * kScanPer;

struct __align__(16) TileRec {
    int32_t m, s, tr, flags;  // flags: 1 continues (full), 2 mark before the tile, 4 mark after it
};

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
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// ============================================================================ count pass
template <int TW>
__global__ void __launch_bounds__(256, 2) daq_count_kernel(const __grid_constant__ KArgs a)
{
    constexpr int NWT = TW / 32, NBT = TW / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char *slot0 = smem;
    uint8_t *abyte = smem + 2 * (size_t)a.slot_bytes;              // 128 bytes
    int32_t *blocksum = reinterpret_cast<int32_t *>(abyte + 128);  // NBT
    int32_t *sarr = blocksum + NBT;                                // TW when needed
    TileInfo *tinfo = reinterpret_cast<TileInfo *>(
        (reinterpret_cast<uintptr_t>(sarr + (a.need_sarr ? TW : 0)) + 15) & ~uintptr_t(15));  // [2]
    uint64_t *bar = reinterpret_cast<uint64_t *>(tinfo + 2);                                  // [2]

    for (int i = tid; i < 32; i += 256) reinterpret_cast<uint32_t *>(abyte)[i] = 0u;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const long long total = a.fill_tile_start[a.n_fills];
    const long long G = gridDim.x;
    const int n_steps = (a.ew + 63) / 64;
    const bool skip_q = (a.flags & DAQ_SKIP_Q) != 0;

    auto start_load = [&](long long tile, int s) {  // thread 0
        TileInfo &T = tinfo[s];
        decode_tile<TW>(a, tile, T, a.fill_tile_start, a.lens);
        trace_stamp(a, tile, 0);
        trace_value(a, tile, 10, sm_id());
        trace_value(a, tile, 11, TW);
        unsigned char *slot = slot0 + (size_t)s * a.slot_bytes;
        if (a.use_tma) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar + s, tile_load_bytes(a));
            issue_tile_load(a, T, slot, bar + s);
        }
        trace_stamp(a, tile, 1);
    };
    if (tid == 0 && (long long)blockIdx.x < total) start_load(blockIdx.x, 0);
    for (long long j = 0;; ++j) {
        const long long tile = blockIdx.x + j * G;
        if (tile >= total) break;
        const int s = (int)(j & 1);
        __syncthreads();  // tinfo[s] is visible; slot s^1 is no longer read
        if (tid == 0 && tile + G < total) start_load(tile + G, s ^ 1);
        const TileInfo T = tinfo[s];
        unsigned char *slot = slot0 + (size_t)s * a.slot_bytes;
        if (a.use_tma) {
            const bool ok = mbar_wait_bounded(bar + s, (uint32_t)((j >> 1) & 1), kWaitLimitNs);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) set_status_bit(a, DAQ_DEV_TIMEOUT);
                return;
            }
        } else {
            plain_tile_load(a, T, slot, tid, 256);
            __syncthreads();
        }
        if (tid == 0) trace_stamp(a, T.tile, 2);
        const uint32_t slot_s = smem_addr(slot);
        for (int it = warp; it < n_steps; it += 8)
            sum_pass_step(a, T, slot_s, it, NBT, abyte, blocksum, sarr, nullptr, lane);
        __syncthreads();
        if (tid == 0) trace_stamp(a, T.tile, 3);
        if (warp == 0) {
            unsigned edges;
            const uint32_t Mt = tile_marks<TW>(a, T, abyte, &edges, lane);
            const Agg agg = words_from_marks<TW>(Mt, edges & 1u, edges >> 1, (int)(T.t_end - T.t0),
                                                 TileWords{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr},
                                                 nullptr, lane);
            if (lane < NWT) a.marks[T.tile * NWT + lane] = Mt;
            if (lane == 0) {
                TileRec r;
                r.m = (int32_t)agg.m;
                r.s = (int32_t)agg.s;
                r.tr = (int32_t)agg.tr;
                r.flags = (agg.full ? 1 : 0) | (int)((edges & 1u) << 1) | (int)((edges >> 1) << 2);
                reinterpret_cast<TileRec *>(a.recs)[T.tile] = r;
                trace_stamp(a, T.tile, 4);
            }
        } else if (!skip_q) {
            q_partial(a, T, blocksum, sarr, tid - 32, 256 - 32);
        }
    }
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

__global__ void __launch_bounds__(kScanThreads) daq_scan_reduce_kernel(const __grid_constant__ KArgs a)
{
    __shared__ Agg warp_tot[kScanThreads / 32];
    const long long total = a.fill_tile_start[a.n_fills];
    const long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanPer;
    const TileRec *recs = reinterpret_cast<const TileRec *>(a.recs);
    Agg v = agg_identity();
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < total) v = combine(v, rec_agg(recs[base + i]));
    Agg tot;
    block_scan_incl(v, warp_tot, &tot);
    if (threadIdx.x == 0) a.blockagg[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) daq_scan_apply_kernel(const __grid_constant__ KArgs a)
{
    __shared__ Agg warp_tot[kScanThreads / 32];
    __shared__ Agg s_incl[kScanThreads];
    __shared__ Agg s_prefix;
    const long long total = a.fill_tile_start[a.n_fills];
    const long long chunk0 = (long long)blockIdx.x * kScanChunk;
    if (chunk0 >= total) return;
    if (threadIdx.x == 0) {
        Agg p = agg_identity();
        for (unsigned b = 0; b < blockIdx.x; ++b) p = combine(p, a.blockagg[b]);
        s_prefix = p;
    }
    const long long base = chunk0 + (long long)threadIdx.x * kScanPer;
    const TileRec *recs = reinterpret_cast<const TileRec *>(a.recs);
    TileRec r[kScanPer];
    Agg v = agg_identity();
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        r[i] = base + i < total ? recs[base + i] : TileRec{0, 0, 0, 1};
        v = combine(v, rec_agg(r[i]));
    }
    Agg blk_tot;
    s_incl[threadIdx.x] = block_scan_incl(v, warp_tot, &blk_tot);
    __syncthreads();
    Agg ex = threadIdx.x == 0 ? s_prefix : combine(s_prefix, s_incl[threadIdx.x - 1]);
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

__device__ __forceinline__ void issue_tile_load_b(const KArgs &a, const TileInfo &T, unsigned char *slot,
                                                  uint64_t *bar)
{
    const int c0 = (int)T.t0;
    const int c1 = (int)(((long long)T.f * a.n_calo + T.c) * a.n_xtal);
    for (int k = 0; k < a.nbox_b; ++k)
        tma_load_2d(slot + (size_t)k * a.box_stride_b, &a.tmap_b, c0 + k * a.boxw_b, c1, bar);
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

template <int TW>
__global__ void __launch_bounds__(256, 2) daq_compact_kernel(const __grid_constant__ KArgs a)
{
    constexpr int NWT = TW / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const long long total = a.fill_tile_start[a.n_fills];
    const TileRec *recs = reinterpret_cast<const TileRec *>(a.recs);
    const TileExcl *exs = reinterpret_cast<const TileExcl *>(a.excl);
    uint32_t phase_bit = 0;
    bool store_pending = false;
    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        if (tid == 0) {
            decode_tile<TW>(a, tile, *tinfo, a.fill_tile_start, a.lens);
            trace_stamp(a, tile, 5);
            if (a.use_tma) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, (uint32_t)a.nbox_b * (uint32_t)X * (uint32_t)a.rs_b);
                issue_tile_load_b(a, *tinfo, slot, bar);
            }
        }
        __syncthreads();
        const TileInfo T = *tinfo;
        if (!a.use_tma) plain_tile_load_b(a, T, slot, tid, 256);
        if (warp == 0) {
            const TileRec r = recs[tile];
            const TileExcl e = exs[tile];
            const uint32_t Mt = lane < NWT ? a.marks[tile * NWT + lane] : 0u;
            const Agg g = words_from_marks<TW>(Mt, (r.flags >> 1) & 1, (r.flags >> 2) & 1, (int)(T.t_end - T.t0),
                                               W, nullptr, lane);
            if (lane == 0) {
                Agg ex;
                ex.m = e.m;
                ex.s = e.s;
                ex.tr = e.tr;
                ex.full = 0;
                ex.poison = 0;
                *s_ex = ex;
                *s_agg = g;
            }
        }
        if (tid == 0 && store_pending) {  // the stage is free once the last bulk store has read it
            bulk_wait_read0();
            store_pending = false;
        }
        if (a.use_tma) {
            const bool ok = mbar_wait_bounded(bar, phase_bit, kWaitLimitNs);
            phase_bit ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) set_status_bit(a, DAQ_DEV_TIMEOUT);
                return;
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
        for (int it = warp; it < (nt + 63) / 64; it += 8) compact_step(a, smem_addr(slot), it, nt, W.m, W.mb, stage,
                                                                        phase, lane);
        __syncthreads();
        if (tid == 0) trace_stamp(a, tile, 7);
        // rows [ex.m, ex.m + agg.m) <- stage bytes [phase, phase + agg.m * 2X)
        long long ge = gs + agg.m * rb;
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
                bulk_s2g(g + a16, stage + phase + (a16 - gs), (uint32_t)(b16 - a16));
                bulk_commit();
                store_pending = true;
            }
            const int n_head = (int)((a16 - gs) >> 1), n_tail = (int)((ge - b16) >> 1);
            if (tid >= 32 && tid < 32 + n_head)
                *reinterpret_cast<uint16_t *>(g + gs + 2 * (tid - 32)) =
                    *reinterpret_cast<const uint16_t *>(stage + phase + 2 * (tid - 32));
            else if (tid >= 64 && tid < 64 + n_tail) {
                const long long o = b16 + 2 * (tid - 64);
                *reinterpret_cast<uint16_t *>(g + o) = *reinterpret_cast<const uint16_t *>(stage + phase + (o - gs));
            }
        }
        if (warp == 0) write_headers<TW>(a, T, W, ex, lane);
        if (tid == 0) trace_stamp(a, tile, 9);
    }
    if (tid == 0 && store_pending) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

}  // namespace daq
