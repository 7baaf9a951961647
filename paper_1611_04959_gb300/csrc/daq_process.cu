// Fused per-fill processing of muon g-2 calorimeter waveforms on sm_103a.
//
// Paper: W. Gohn, arXiv:1611.04959, Sec. 3 and Table 2.  The eight kernels of
// Table 2 (pedestal, threshold, pre/post samples, merge, save islands, sum,
// Q decimation, fill-by-fill sum) become two launches:
//
//   daq_prepare_kernel  pedestals (Table 2 row 1) for every (fill, calo,
//                       crystal), the per-fill tile plan, and the reset of the
//                       scan workspace;
//   a tile kernel       one pass over the samples.  Tiles of TW samples of one
//                       calorimeter-fill are taken in order (atomic ticket); the
//                       crystal rows of a tile plus a halo are bulk-copied into
//                       shared memory, and from there the kernel sums crystals
//                       and subtracts pedestals (row 6), tests the threshold
//                       (row 2), widens crossings by the pre/post windows
//                       (row 3), finds island starts and ends (row 4), takes its
//                       global pool-row and island offsets from a single-pass
//                       decoupled look-back scan over tiles, writes island
//                       records and time-major pool rows (row 5), and adds
//                       decimated partial sums into the int64 Q histograms
//                       (rows 7-8).
//
// Two tile kernels implement the same steps (daq_steps.cuh):
//   daq_pipe_kernel  the default: one persistent CTA per SM whose warps have
//                    fixed roles (bulk-load producer, crystal-sum/staging warps,
//                    window/merge warp, look-back warp, writer warps) handing
//                    tiles to each other through mbarriers, so loads, scan
//                    waits and stores of different tiles overlap;
//   daq_tile_kernel  the plain form: every step of a tile in sequence by one
//                    CTA (launched one CTA per tile, or persistent).
//
// Every quantity is an integer, so results do not depend on kernel, tile
// size, grid size or the order in which tiles run.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "daq.h"
#include "daq_device.cuh"
#include "daq_steps.cuh"
#include "daq_twopass.cuh"
#include "daq_stream.cuh"
#include "daq_park.cuh"

namespace daq {

constexpr int kThreads = 256;  // prepare kernel and plain tile kernel
constexpr int kWarps = kThreads / 32;

// Stage row pitch: P words, P the first odd number >= ceil(n_xtal / 2).  A warp's
// staging store writes one word into each of 32 rows 2 apart, which an odd P
// spreads over 16 banks (2-way conflicts at worst).
static int stage_row_bytes(int X)
{
    int P = (X + 1) / 2;
    if (!(P & 1)) ++P;
    return 4 * P;
}

// Workspace layout (byte offsets from the workspace base).
struct WsLayout {
    size_t ticket, fts, lens, ptot, status, marks, recs, excl, scan_status, total;
};

static WsLayout ws_layout(int64_t n_fills, int64_t n_calo, int64_t max_tiles)
{
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    WsLayout w;
    w.ticket = 0;
    w.fts = up(512);  // [0, 16) ticket; 128 and 256: counters of the single-launch form; 384: scan ticket
    w.lens = up(w.fts + sizeof(long long) * (size_t)(n_fills + 1));
    w.ptot = up(w.lens + sizeof(int32_t) * (size_t)(n_fills > 0 ? n_fills : 1));
    w.status = up(w.ptot + sizeof(int32_t) * (size_t)(n_fills * n_calo > 0 ? n_fills * n_calo : 1));
    const size_t nt = (size_t)(max_tiles > 0 ? max_tiles : 1);
    w.marks = up(w.status + sizeof(TileStatus) * nt);
    w.recs = up(w.marks + sizeof(uint32_t) * (size_t)(kMaxTileWords) * nt);
    w.excl = up(w.recs + sizeof(TileRec) * nt);
    w.scan_status = up(w.excl + sizeof(TileExcl) * nt);
    w.total = up(w.scan_status + sizeof(TileStatus) * ((nt + kScanChunk - 1) / kScanChunk));
    return w;
}

__device__ __forceinline__ long long floor_div_ll(long long a, long long b)
{
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// ============================================================================ prepare
// Grid-stride over calorimeter-fills.  Block 0 also zeroes counts, validates
// fill lengths and writes the tile plan.  Every block zeroes part of the
// tile-status array.
__global__ void __launch_bounds__(kThreads) daq_prepare_kernel(KArgs a, int tw)
{
    pdl_trigger();  // the count kernel's CTAs may become resident; they wait for this kernel to finish
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ long long s_warp[kWarps];
    __shared__ long long s_carry;
    __shared__ long long s_ped[kWarps];

    if (a.mode == kModeFused) {  // records carry a valid bit; counters restart at 0
        uint4 *rc = reinterpret_cast<uint4 *>(a.recs);
        for (long long i = (long long)blockIdx.x * kThreads + tid; i < a.max_tiles; i += (long long)gridDim.x * kThreads)
            rc[i] = make_uint4(0u, 0u, 0u, 0u);
        if (blockIdx.x == 0 && tid < 2) a.fctr[16 * tid] = 0ull;
    } else if (a.mode != kModeTwoPass) {  // scan state of the single-pass kernels
        uint4 *st = reinterpret_cast<uint4 *>(a.status);
        const long long n16 = a.max_tiles * (long long)(sizeof(TileStatus) / 16);
        for (long long i = (long long)blockIdx.x * kThreads + tid; i < n16; i += (long long)gridDim.x * kThreads)
            st[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {  // the chained scan's block states and ticket
        uint4 *st = reinterpret_cast<uint4 *>(a.scan_status);
        const long long n16 = (a.max_tiles + kScanChunk - 1) / kScanChunk;
        for (long long i = (long long)blockIdx.x * kThreads + tid; i < n16; i += (long long)gridDim.x * kThreads)
            st[i] = make_uint4(0u, 0u, 0u, 0u);
        if (blockIdx.x == 0 && tid == 0) *a.scan_ticket = 0u;
    }

    if (blockIdx.x == 0) {
        if (tid == 0) {
            *a.ticket = 0u;
            a.counts[0] = 0;
            a.counts[1] = 0;
            a.counts[2] = 0;
            a.counts[3] = 0;
            s_carry = 0;
        }
        __syncthreads();
        int bad = 0;
        for (int f0 = 0; f0 < a.n_fills; f0 += kThreads) {
            const int f = f0 + tid;
            long long tiles = 0;
            if (f < a.n_fills) {
                long long len = a.fill_len ? (long long)a.fill_len[f] : a.n_samples;
                if (len < 0 || len > a.n_samples) {
                    bad = 1;
                    len = len < 0 ? 0 : a.n_samples;
                }
                a.lens[f] = (int32_t)len;
                tiles = ((len + tw - 1) / tw) * (long long)a.n_calo;
            }
            long long tot;
            const long long ex = warp_excl_scan_add<long long>(tiles, lane, tot);
            if (lane == 0) s_warp[warp] = tot;
            __syncthreads();
            long long before = s_carry;
            for (int w = 0; w < warp; ++w) before += s_warp[w];
            if (f < a.n_fills) a.fill_tile_start[f] = before + ex;
            __syncthreads();
            if (tid == kThreads - 1) {
                long long all = 0;
                for (int w = 0; w < kWarps; ++w) all += s_warp[w];
                s_carry += all;
            }
            __syncthreads();
        }
        if (tid == 0) a.fill_tile_start[a.n_fills] = s_carry;
        if (__syncthreads_or(bad) && tid == 0) set_status_bit(a, DAQ_DEV_BAD_FILL_LEN);
    }

    // pedestals: warp per crystal, block per calorimeter-fill
    const long long n_cf = (long long)a.n_fills * a.n_calo;
    for (long long cf = blockIdx.x; cf < n_cf; cf += gridDim.x) {
        const int f = (int)(cf / a.n_calo);
        long long len = a.fill_len ? (long long)a.fill_len[f] : a.n_samples;
        len = len < 0 ? 0 : (len > a.n_samples ? a.n_samples : len);
        const long long n = len < a.ped_samples ? len : a.ped_samples;
        long long ptot_part = 0;
        auto finish = [&](int x, long long sum) {  // warp sum of crystal x's window -> its pedestal
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(kFull, sum, d);
            const long long p = n > 0 ? floor_div_ll(sum + n / 2, n) : 0;
            if (lane == 0 && a.ped_out && !(a.flags & DAQ_SKIP_ISLANDS)) a.ped_out[cf * a.n_xtal + x] = (int32_t)p;
            ptot_part += p;
        };
        if (n <= 256 && (a.n_samples & 7) == 0 && (reinterpret_cast<uintptr_t>(a.samples) & 15) == 0) {
            // lane L sums samples [8L, 8L + 8) of the window with one 16-byte load per
            // crystal; the loads of kPedX crystals are in flight at once
            constexpr int kPedX = 8;
            for (int x0 = warp; x0 < a.n_xtal; x0 += kWarps * kPedX) {
                int4 v[kPedX];
#pragma unroll
                for (int k = 0; k < kPedX; ++k) {
                    const int x = x0 + k * kWarps;
                    v[k] = make_int4(0, 0, 0, 0);
                    if (x < a.n_xtal && 8 * lane < n)
                        v[k] = __ldg(reinterpret_cast<const int4 *>(a.samples + (cf * a.n_xtal + x) * a.n_samples) + lane);
                }
#pragma unroll
                for (int k = 0; k < kPedX; ++k) {
                    const int x = x0 + k * kWarps;
                    if (x >= a.n_xtal) break;
                    const uint32_t w[4] = {(uint32_t)v[k].x, (uint32_t)v[k].y, (uint32_t)v[k].z, (uint32_t)v[k].w};
                    long long sum = 0;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int16_t val = (int16_t)((w[j >> 1] >> (16 * (j & 1))) & 0xffffu);
                        if (8 * lane + j < n) sum += val;
                    }
                    finish(x, sum);
                }
            }
        } else {
            for (int x = warp; x < a.n_xtal; x += kWarps) {
                const int16_t *row = a.samples + (cf * a.n_xtal + x) * a.n_samples;
                long long sum = 0;
                for (long long t = lane; t < n; t += 32) sum += row[t];
                finish(x, sum);
            }
        }
        if (lane == 0) s_ped[warp] = ptot_part;
        __syncthreads();
        if (tid == 0) {
            long long t = 0;
            for (int w = 0; w < kWarps; ++w) t += s_ped[w];
            a.ptot[cf] = (int32_t)t;
        }
        __syncthreads();
    }
}

// ============================================================================ plain tile kernel
template <int TW>
__global__ void __launch_bounds__(kThreads, 2) daq_tile_kernel(const __grid_constant__ KArgs a)
{
    constexpr int NWT = TW / 32;
    constexpr int NBT = TW / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    unsigned char *tbuf = smem;                                    // tile slot (nbox boxes)
    unsigned char *stage = tbuf + a.slot_bytes;                    // TW rows of srow bytes + 32
    const int stage_bytes = ((TW * a.srow + 32) + 15) & ~15;
    uint8_t *abyte = stage + stage_bytes;                          // 128 bytes
    int32_t *blocksum = reinterpret_cast<int32_t *>(abyte + 128);  // NBT
    int32_t *sarr = blocksum + NBT;                                // TW when needed
    uint32_t *wm = reinterpret_cast<uint32_t *>(sarr + (a.need_sarr ? TW : 0));
    TileWords W{wm, wm + NWT, wm + 2 * NWT, reinterpret_cast<int32_t *>(wm + 3 * NWT),
                reinterpret_cast<int32_t *>(wm + 4 * NWT), reinterpret_cast<int32_t *>(wm + 5 * NWT)};
    int16_t *rowtab = reinterpret_cast<int16_t *>(wm + 6 * NWT);  // TW
    TileInfo *tinfo = reinterpret_cast<TileInfo *>((reinterpret_cast<uintptr_t>(rowtab + TW) + 15) & ~uintptr_t(15));
    Agg *s_agg = reinterpret_cast<Agg *>(tinfo + 1);  // [0] aggregate, [1] exclusive prefix
    uint64_t *bar = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(s_agg + 2) + 15) & ~uintptr_t(15));

    for (int i = tid; i < 32; i += kThreads) reinterpret_cast<uint32_t *>(abyte)[i] = 0u;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    const uint32_t tile_s = smem_addr(tbuf);
    const int n_steps = (a.ew + 63) / 64;
    const bool skip_isl = (a.flags & DAQ_SKIP_ISLANDS) != 0;
    const long long total = a.fill_tile_start[a.n_fills];

    uint32_t phase = 0;
    for (;;) {
        if (tid == 0) {
            const long long tk = (long long)atomicAdd(a.ticket, 1u);
            decode_tile<TW>(a, tk, *tinfo, a.fill_tile_start, a.lens);
        }
        __syncthreads();
        const TileInfo T = *tinfo;
        if (T.tile < 0) break;
        if (tid == 0) {
            trace_stamp(a, T.tile, 0);
            trace_value(a, T.tile, 10, sm_id());
            trace_value(a, T.tile, 11, TW);
        }

        if (a.use_tma) {
            if (tid == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, tile_load_bytes(a));
                issue_tile_load(a, T, tbuf, bar);
                trace_stamp(a, T.tile, 1);
            }
            const bool ok = mbar_wait_bounded(bar, phase, kWaitLimitNs);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) set_status_bit(a, DAQ_DEV_TIMEOUT);
                mbar_wait_bounded(bar, phase ^ 1u, kWaitLimitNs);
                return;
            }
        } else {
            plain_tile_load(a, T, tbuf, tid, kThreads);
            __syncthreads();
        }

        if (tid == 0) trace_stamp(a, T.tile, 2);
        for (int it = warp; it < n_steps; it += kWarps)
            sum_pass_step(a, T, tile_s, it, NBT, abyte, blocksum, sarr, skip_isl ? nullptr : stage, lane);
        __syncthreads();
        if (tid == 0) trace_stamp(a, T.tile, 3);

        if (warp == 0) {
            const Agg agg = tile_bits<TW>(a, T, abyte, W, rowtab, lane);
            if (lane == 0) {
                trace_stamp(a, T.tile, 4);
                trace_stamp(a, T.tile, 5);
            }
            Agg excl = agg_identity();
            if (T.tile > 0) {
                if (lane == 0) publish(a.status, T.tile, false, agg);
                excl = look_back(a, T.tile, lane);
            }
            if (lane == 0) {
                publish(a.status, T.tile, true, combine(excl, agg));
                s_agg[0] = agg;
                s_agg[1] = excl;
                trace_stamp(a, T.tile, 6);
            }
        } else {
            if (!(a.flags & DAQ_SKIP_Q)) q_partial(a, T, blocksum, sarr, tid - 32, kThreads - 32);
        }
        __syncthreads();

        const Agg agg = s_agg[0], excl = s_agg[1];
        if (tid == 0) {
            trace_stamp(a, T.tile, 7);
            trace_stamp(a, T.tile, 8);
        }
        if (!excl.poison && !skip_isl) {
            copy_out(a, stage, rowtab, excl, agg, tid, kThreads, TW);
            if (warp == 0) write_headers<TW>(a, T, W, excl, lane);
        }
        if (tid == 0) trace_stamp(a, T.tile, 9);
        if (tid == 0 && T.tile == total - 1) write_counts(a, T.tile, combine(excl, agg));
    }
}

// ============================================================================ pipelined tile kernel
// Warp roles (one persistent CTA per SM):
constexpr int kPipeProducer = 0;           // tickets, decode, bulk loads
constexpr int kPipeCompute0 = 1;           // crystal sums, threshold bits, staging
constexpr int kPipeNCompute = 8;
constexpr int kPipeBits = kPipeCompute0 + kPipeNCompute;  // windows, merge, aggregate
constexpr int kPipeLook = kPipeBits + 1;                  // decoupled look-back (alternate tiles)
constexpr int kPipeNLook = 2;
constexpr int kPipeWriter0 = kPipeLook + kPipeNLook;      // Q, pool rows, island records
constexpr int kPipeNWriter = 4;
constexpr int kPipeWarps = kPipeWriter0 + kPipeNWriter;
constexpr int kPipeThreads = 32 * kPipeWarps;
constexpr int kNIn = 2;   // input tile slots
constexpr int kNOut = 2;  // stage slots
constexpr int kNMeta = 4; // tiles in flight per CTA
constexpr int kPlanCache = 64;  // fills whose tile plan is cached in shared memory

template <int TW> struct PipeMeta {
    TileInfo T;
    Agg agg, excl;
    uint8_t abyte[128];
    int32_t blocksum[TW / 8];
    uint32_t wm[TW / 32], ws[TW / 32], we[TW / 32];
    int32_t wmb[TW / 32], wsb[TW / 32], wls[TW / 32];
    int16_t rowtab[TW];
};

// mbarrier indices
enum {
    kBarInFull = 0,
    kBarInEmpty = kBarInFull + kNIn,
    kBarOutFull = kBarInEmpty + kNIn,
    kBarOutEmpty = kBarOutFull + kNOut,
    kBarBits = kBarOutEmpty + kNOut,
    kBarWords = kBarBits + kNMeta,
    kBarAgg = kBarWords + kNMeta,
    kBarExcl = kBarAgg + kNMeta,
    kBarMetaFree = kBarExcl + kNMeta,
    kNBars = kBarMetaFree + kNMeta
};

// Bounded wait that also returns early once any CTA has flagged a timeout.
__device__ __forceinline__ bool pipe_wait(const KArgs &a, uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if ((i & 3u) == 3u) {
            if (global_ns() - t0 > kWaitLimitNs) {
                set_status_bit(a, DAQ_DEV_TIMEOUT);
                return false;
            }
            if (aborted(a)) return false;
        }
    }
}

template <int TW> static size_t pipe_smem_bytes(int X, int slot_bytes, int rs, int need_sarr)
{
    size_t b = (size_t)kNIn * slot_bytes;
    b += (size_t)kNOut * (size_t)(((TW * stage_row_bytes(X) + 32) + 15) & ~15);
    b += (size_t)kNMeta * ((sizeof(PipeMeta<TW>) + 15) & ~size_t(15));
    b += need_sarr ? (size_t)kNMeta * TW * 4 : 0;
    b += (size_t)kNBars * 8 + 16;
    b += (size_t)(kPlanCache + 1) * 8 + (size_t)kPlanCache * 4 + 16;
    b += 16;  // end index
    return (b + 127) & ~size_t(127);
}

template <int TW>
__global__ void __launch_bounds__(kPipeThreads, 1) daq_pipe_kernel(const __grid_constant__ KArgs a)
{
    constexpr int NBT = TW / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int stage_bytes = ((TW * a.srow + 32) + 15) & ~15;
    constexpr size_t meta_bytes = (sizeof(PipeMeta<TW>) + 15) & ~size_t(15);

    unsigned char *in0 = smem;
    unsigned char *out0 = in0 + (size_t)kNIn * a.slot_bytes;
    unsigned char *meta0 = out0 + (size_t)kNOut * stage_bytes;
    int32_t *sarr0 = reinterpret_cast<int32_t *>(meta0 + kNMeta * meta_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(sarr0 + (a.need_sarr ? kNMeta * TW : 0)) + 15) & ~uintptr_t(15));
    long long *plan_fts = reinterpret_cast<long long *>(bars + kNBars);
    int32_t *plan_lens = reinterpret_cast<int32_t *>(plan_fts + kPlanCache + 1);
    // iteration at which the producer found no more tiles (read by the look-back warps)
    volatile long long *s_end = reinterpret_cast<volatile long long *>(
        (reinterpret_cast<uintptr_t>(plan_lens + kPlanCache) + 15) & ~uintptr_t(15));
    if (tid == 0) *s_end = 0x7fffffffffffffffll;
    const bool cached = a.n_fills <= kPlanCache;
    if (cached) {
        for (int f = tid; f <= a.n_fills; f += kPipeThreads) plan_fts[f] = a.fill_tile_start[f];
        for (int f = tid; f < a.n_fills; f += kPipeThreads) plan_lens[f] = a.lens[f];
    }
    const long long *fts = cached ? plan_fts : a.fill_tile_start;
    const int32_t *lens = cached ? plan_lens : a.lens;
    auto meta = [&](int m) { return reinterpret_cast<PipeMeta<TW> *>(meta0 + m * meta_bytes); };
    auto sarr = [&](int m) { return sarr0 + (a.need_sarr ? m * TW : 0); };
    auto words = [&](int m) {
        PipeMeta<TW> *M = meta(m);
        return TileWords{M->wm, M->ws, M->we, M->wmb, M->wsb, M->wls};
    };

    for (int m = 0; m < kNMeta; ++m)
        for (int i = tid; i < 32; i += kPipeThreads) reinterpret_cast<uint32_t *>(meta(m)->abyte)[i] = 0u;
    if (tid == 0) {
        for (int s = 0; s < kNIn; ++s) {
            mbar_init(bars + kBarInFull + s, 1);
            mbar_init(bars + kBarInEmpty + s, kPipeNCompute);
        }
        for (int o = 0; o < kNOut; ++o) {
            mbar_init(bars + kBarOutFull + o, kPipeNCompute);
            mbar_init(bars + kBarOutEmpty + o, kPipeNWriter);
        }
        for (int m = 0; m < kNMeta; ++m) {
            mbar_init(bars + kBarBits + m, kPipeNCompute);
            mbar_init(bars + kBarWords + m, 1);
            mbar_init(bars + kBarAgg + m, 1);
            mbar_init(bars + kBarExcl + m, 1);
            mbar_init(bars + kBarMetaFree + m, kPipeNWriter);
        }
        fence_mbar_init();
    }
    __syncthreads();

    const long long total = a.fill_tile_start[a.n_fills];
    const bool skip_isl = (a.flags & DAQ_SKIP_ISLANDS) != 0;

    if (warp == kPipeProducer) {
        // ------------------------------------------------------------ producer
        uint32_t pending = 0, pend_parity = 0;  // per input slot: load issued, its phase parity
        for (long long i = 0;; ++i) {
            const int s = (int)(i % kNIn), m = (int)(i % kNMeta);
            if (i >= kNIn && !pipe_wait(a, bars + kBarInEmpty + s, (uint32_t)((i / kNIn - 1) & 1))) break;
            if (i >= kNMeta && !pipe_wait(a, bars + kBarMetaFree + m, (uint32_t)((i / kNMeta - 1) & 1))) break;
            pending &= ~(1u << s);
            PipeMeta<TW> *M = meta(m);
            int valid = 0;
            const unsigned long long t_free = global_ns();
            if (lane == 0) {
                const long long tk = (long long)atomicAdd(a.ticket, 1u);
                valid = decode_tile<TW>(a, tk, M->T, fts, lens);
                if (valid) trace_value(a, tk, 15, t_free);
            }
            valid = __shfl_sync(kFull, valid, 0);
            __syncwarp();
            if (!valid) {
                if (lane == 0) {
                    *s_end = i;
                    mbar_arrive(bars + kBarInFull + s);
                }
                break;
            }
            const TileInfo T = M->T;
            if (lane == 0) {
                trace_stamp(a, T.tile, 0);
                trace_value(a, T.tile, 10, sm_id());
                trace_value(a, T.tile, 11, TW);
            }
            unsigned char *slot = in0 + (size_t)s * a.slot_bytes;
            if (a.use_tma) {
                if (lane == 0) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(bars + kBarInFull + s, tile_load_bytes(a));
                    issue_tile_load(a, T, slot, bars + kBarInFull + s);
                    trace_stamp(a, T.tile, 1);
                }
                __syncwarp();
                pending |= 1u << s;
                pend_parity = (pend_parity & ~(1u << s)) | ((uint32_t)((i / kNIn) & 1) << s);
            } else {
                plain_tile_load(a, T, slot, lane, 32);
                __syncwarp();
                if (lane == 0) mbar_arrive(bars + kBarInFull + s);
            }
        }
        // bulk copies still in flight land before this CTA may exit
        for (int s = 0; s < kNIn; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(bars + kBarInFull + s, (pend_parity >> s) & 1u, kWaitLimitNs);
    } else if (warp >= kPipeCompute0 && warp < kPipeCompute0 + kPipeNCompute) {
        // ------------------------------------------------------------ crystal sums + staging
        const int cw = warp - kPipeCompute0;
        const int n_steps = (a.ew + 63) / 64;
        for (long long i = 0;; ++i) {
            const int s = (int)(i % kNIn), m = (int)(i % kNMeta), o = (int)(i % kNOut);
            if (i >= kNOut && !pipe_wait(a, bars + kBarOutEmpty + o, (uint32_t)((i / kNOut - 1) & 1))) break;
            if (!pipe_wait(a, bars + kBarInFull + s, (uint32_t)((i / kNIn) & 1))) break;
            PipeMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) {
                __syncwarp();
                if (lane == 0) mbar_arrive(bars + kBarBits + m);
                break;
            }
            if (cw == 0 && lane == 0) trace_stamp(a, T.tile, 2);
            const uint32_t slot_s = smem_addr(in0 + (size_t)s * a.slot_bytes);
            unsigned char *stage = skip_isl ? nullptr : out0 + (size_t)o * stage_bytes;
            for (int it = cw; it < n_steps; it += kPipeNCompute)
                sum_pass_step(a, T, slot_s, it, NBT, M->abyte, M->blocksum, sarr(m), stage, lane);
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bars + kBarBits + m);
                mbar_arrive(bars + kBarInEmpty + s);
                mbar_arrive(bars + kBarOutFull + o);
                if (cw == 0) {
                    trace_stamp(a, T.tile, 3);
                    trace_stamp(a, T.tile, 7);
                }
            }
        }
    } else if (warp == kPipeBits) {
        // ------------------------------------------------------------ windows + merge
        for (long long i = 0;; ++i) {
            const int m = (int)(i % kNMeta);
            if (!pipe_wait(a, bars + kBarBits + m, (uint32_t)((i / kNMeta) & 1))) break;
            PipeMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) {
                if (lane == 0) {
                    mbar_arrive(bars + kBarWords + m);
                    mbar_arrive(bars + kBarAgg + m);
                }
                break;
            }
            const Agg agg = tile_bits<TW>(a, T, M->abyte, words(m), M->rowtab, lane);
            if (lane == 0) {
                trace_stamp(a, T.tile, 4);
                M->agg = agg;
                if (T.tile > 0) publish(a.status, T.tile, false, agg);
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bars + kBarWords + m);
                mbar_arrive(bars + kBarAgg + m);
            }
        }
    } else if (warp >= kPipeLook && warp < kPipeLook + kPipeNLook) {
        // ------------------------------------------------------------ decoupled look-back
        for (long long i = warp - kPipeLook;; i += kPipeNLook) {
            const int m = (int)(i % kNMeta);
            // the other look-back warp may own the end marker: stop once it is past
            bool ready = false, done = false;
            const uint64_t t0 = global_ns();
            for (uint32_t k = 0; !ready && !done; ++k) {
                ready = mbar_try_wait_sleep(bars + kBarAgg + m, (uint32_t)((i / kNMeta) & 1), 2000u);
                if (!ready && *s_end < i) done = true;
                if (!ready && (k & 15u) == 15u) {
                    if (global_ns() - t0 > kWaitLimitNs) {
                        set_status_bit(a, DAQ_DEV_TIMEOUT);
                        done = true;
                    } else if (aborted(a)) {
                        done = true;
                    }
                }
            }
            if (!ready) break;
            PipeMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) {
                if (lane == 0) mbar_arrive(bars + kBarExcl + m);
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
            if (lane == 0) mbar_arrive(bars + kBarExcl + m);
        }
    } else {
        // ------------------------------------------------------------ writers
        const int gt = tid - 32 * kPipeWriter0;
        const int nthr = 32 * kPipeNWriter;
        for (long long i = 0;; ++i) {
            const int m = (int)(i % kNMeta), o = (int)(i % kNOut);
            if (!pipe_wait(a, bars + kBarExcl + m, (uint32_t)((i / kNMeta) & 1))) break;
            PipeMeta<TW> *M = meta(m);
            const TileInfo T = M->T;
            if (T.tile < 0) break;
            const Agg agg = M->agg, excl = M->excl;
            if (gt == 0) trace_stamp(a, T.tile, 8);
            if (!(a.flags & DAQ_SKIP_Q)) q_partial(a, T, M->blocksum, sarr(m), gt, nthr);
            if (!pipe_wait(a, bars + kBarOutFull + o, (uint32_t)((i / kNOut) & 1))) break;
            if (gt == 0) trace_stamp(a, T.tile, 12);
            if (!excl.poison && !skip_isl) {
                copy_out(a, out0 + (size_t)o * stage_bytes, M->rowtab, excl, agg, gt, nthr, TW);
                if (gt == 0) trace_stamp(a, T.tile, 13);
                if (warp == kPipeWriter0) write_headers<TW>(a, T, words(m), excl, lane);
            }
            if (gt == 0 && T.tile == total - 1) write_counts(a, T.tile, combine(excl, agg));
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bars + kBarOutEmpty + o);
                mbar_arrive(bars + kBarMetaFree + m);
                if (gt == 0) trace_stamp(a, T.tile, 9);
            }
        }
    }
}

// ============================================================================ host side
static size_t plain_smem_bytes(int tw, int X, int slot_bytes, int rs, int need_sarr)
{
    size_t b = (size_t)slot_bytes + (size_t)tw * 2;  // tile slot, row table
    b += (size_t)(((tw * stage_row_bytes(X) + 32) + 15) & ~15);
    b += 128;
    b += (size_t)(tw / 8) * 4;
    b += need_sarr ? (size_t)tw * 4 : 0;
    b += (size_t)(tw / 32) * 4 * 6;
    b += 16 + sizeof(TileInfo) + 2 * sizeof(Agg) + 16 + 8;
    return (b + 127) & ~size_t(127);
}

static size_t stream_smem(int tw, int X, int slot_bytes, int need_sarr, int nm, int ns)
{
    switch (tw) {
    case 128: return StreamSmem<128>(X, slot_bytes, need_sarr, nm, ns).total;
    case 224: return StreamSmem<224>(X, slot_bytes, need_sarr, nm, ns).total;
    default: return StreamSmem<448>(X, slot_bytes, need_sarr, nm, ns).total;
    }
}

static size_t park_smem(int tw, int X, int slot_bytes, int need_sarr, int nm, int nc, int np)
{
    switch (tw) {
    case 128: return ParkSmem<128>(X, slot_bytes, need_sarr, nm, nc, np).total;
    case 224: return ParkSmem<224>(X, slot_bytes, need_sarr, nm, nc, np).total;
    default: return ParkSmem<448>(X, slot_bytes, need_sarr, nm, nc, np).total;
    }
}

static size_t pipe_smem(int tw, int X, int slot_bytes, int rs, int need_sarr)
{
    switch (tw) {
    case 128: return pipe_smem_bytes<128>(X, slot_bytes, rs, need_sarr);
    case 224: return pipe_smem_bytes<224>(X, slot_bytes, rs, need_sarr);
    case 448: return pipe_smem_bytes<448>(X, slot_bytes, rs, need_sarr);
    default: return pipe_smem_bytes<960>(X, slot_bytes, rs, need_sarr);
    }
}

struct DeviceInfo {
    int sms = 0;
    int smem_optin = 0;
};

static DeviceInfo device_info(int dev)
{
    static std::mutex mu;
    static DeviceInfo cache[64];
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64) return DeviceInfo{};
    if (cache[dev].sms == 0) {
        cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&cache[dev].smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return cache[dev];
}

// Shared memory one CTA may use, for planning before any device is queried
// (GB300: 227 KB).
constexpr int kSmemBudget = 227 * 1024;
constexpr int kSmemPerSM = 228 * 1024;         // shared memory of one SM
constexpr int kSmemPerBlockReserved = 1024;    // reserved by the system for each resident CTA
// Single-launch form: default and least distance (tiles) the count role may
// run ahead of the compact role.  The least is the scanner's round (one block
// of tiles), below which the roles could wait on each other forever.
constexpr int64_t kFusedLagTiles = 1024;
constexpr int64_t kFusedMinLag = 2 * kCountThreads;

struct Plan {
    int tw, hl, hr, ew, rs, boxw, nbox, box_stride, slot_bytes, need_sarr, mode;
    int halo_free;  // two-pass form: the count pass loads the tile proper only
    int boxw_b, nbox_b, box_stride_b, slot_bytes_b, rs_b;  // compact pass (two-pass mode)
    size_t smem, smem_b;                                   // tile (or count) kernel, compact kernel
    int str_meta, str_stages;                              // streaming / single-read forms: tile records, row stages per CTA
    int pk_slots, pk_cols;                                 // single-read form: park slots, Tensor Memory columns per slot
    int count_ns;                                          // two-pass form: tile slots of the count kernel (2 or 3)
    int64_t max_tiles;
    int64_t ws_tiles;  // tiles the workspace is laid out for: also covers the two-pass plan a call may fall back to
};

// Box geometry of `width` samples for the compact pass: nbox boxes of boxw <=
// 248 samples, boxw a multiple of 8.  The compact pass reads along rows, so
// any row pitch is conflict-free; boxes that split the tile exactly read no
// column of the next tile.  (Boxes of one 64-sample step each, which let a
// sparse tile load only its marked steps, cost the dense full fill 16% in the
// compact kernel: seven narrow boxes move the same bytes in 128-byte rows.)
static void box_geometry(int width, int X, int *nbox, int *boxw, int *box_stride)
{
    *nbox = (width + 247) / 248;
    const int bw = (((width + *nbox - 1) / *nbox) + 7) & ~7;
    *boxw = bw;
    *box_stride = (X * 2 * bw + 127) & ~127;
}

static size_t count_smem_bytes(int tw, int slot_bytes, int need_sarr)
{
    return CountSmem::total(slot_bytes, tw, need_sarr);
}

static size_t compact_smem_bytes(int tw, int X, int slot_bytes_b)
{
    size_t b = (size_t)slot_bytes_b + (size_t)(((tw * 2 * X + 32) + 15) & ~15) + (size_t)(tw / 32) * 4 * 6;
    b += 16 + sizeof(TileInfo) + 2 * sizeof(Agg) + 8 + 8 * (kPlanSmem + 1) + 4 * kPlanSmem + 32;
    return (b + 127) & ~size_t(127);
}

// Extended tile = nbox TMA boxes of boxw samples: boxw <= 248 and an odd
// multiple of 8, so a box row (2 boxw bytes) is an odd multiple of 16 bytes.
static void plan_geometry(Plan *pl, int tw, int pre, int post, int X, bool halo_free = false)
{
    pl->tw = tw;
    pl->hl = (post + 1 + 7) & ~7;
    pl->hr = (pre + 1 + 7) & ~7;
    pl->ew = pl->hl + tw + pl->hr;
    pl->nbox = (pl->ew + 247) / 248;
    int boxw = (((pl->ew + pl->nbox - 1) / pl->nbox) + 7) & ~7;
    if (((boxw / 8) & 1) == 0) boxw += 8;
    pl->boxw = boxw;
    pl->rs = 2 * boxw;
    pl->box_stride = (X * pl->rs + 127) & ~127;
    pl->slot_bytes = pl->nbox * pl->box_stride;
    box_geometry(tw, X, &pl->nbox_b, &pl->boxw_b, &pl->box_stride_b);
    pl->rs_b = 2 * pl->boxw_b;
    pl->slot_bytes_b = pl->nbox_b * pl->box_stride_b;
    pl->halo_free = halo_free;
    if (pl->halo_free) {  // the count pass reads the same boxes as the compact pass
        pl->hl = pl->hr = 0;
        pl->ew = tw;
        pl->nbox = pl->nbox_b;
        pl->boxw = pl->boxw_b;
        pl->rs = pl->rs_b;
        pl->box_stride = pl->box_stride_b;
        pl->slot_bytes = pl->slot_bytes_b;
    }
    pl->smem_b = 0;
    if (pl->mode == kModeStream) {
        // two row stages if they fit, then as many tile records as fit (a
        // multiple of 4: four look-back warps take turns)
        const size_t budget = (size_t)kSmemBudget - 1024;  // static shared memory of the kernel
        pl->str_stages = kStrMaxStages;
        pl->str_meta = kStrMaxMeta;
        for (;;) {
            if (stream_smem(tw, X, pl->slot_bytes, pl->need_sarr, pl->str_meta, pl->str_stages) <= budget) break;
            if (pl->str_meta > 4) pl->str_meta -= 4;
            else if (pl->str_stages > 1) {
                pl->str_stages -= 1;
                pl->str_meta = kStrMaxMeta;
            } else break;  // does not fit: make_plan tries a narrower tile
        }
        pl->smem = stream_smem(tw, X, pl->slot_bytes, pl->need_sarr, pl->str_meta, pl->str_stages);
    } else if (pl->mode == kModePark) {
        // two out-stages if they fit, else one; then as many tile records as
        // fit (a multiple of 4); park slots: as many as the Tensor Memory
        // holds, at most one per tile record
        const size_t budget = (size_t)kSmemBudget - 1024;
        pl->pk_cols = park_slot_cols(pl->ew, X);
        pl->str_stages = kPkMaxOut;
        pl->str_meta = kPkMaxMeta;
        auto slots = [&] { return std::max(1, std::min({kPkMaxPark, kPkCols / pl->pk_cols, pl->str_meta})); };
        for (;;) {
            pl->pk_slots = slots();
            if (park_smem(tw, X, pl->slot_bytes, pl->need_sarr, pl->str_meta, pl->str_stages, pl->pk_slots) <= budget)
                break;
            if (pl->str_meta > 4) pl->str_meta -= 4;
            else if (pl->str_stages > 1) {
                pl->str_stages -= 1;
                pl->str_meta = kPkMaxMeta;
            } else break;  // does not fit: make_plan tries a narrower tile
        }
        pl->pk_slots = slots();
        pl->smem = park_smem(tw, X, pl->slot_bytes, pl->need_sarr, pl->str_meta, pl->str_stages, pl->pk_slots);
        if (pl->pk_cols > kPkCols) pl->smem = (size_t)-1;  // cannot park a tile
    } else if (pl->mode == kModePipelined) {
        pl->smem = pipe_smem(tw, X, pl->slot_bytes, pl->rs, pl->need_sarr);
    } else if (pl->mode == kModePlain) {
        pl->smem = plain_smem_bytes(tw, X, pl->slot_bytes, pl->rs, pl->need_sarr);
    } else {
        pl->smem = count_smem_bytes(tw, pl->slot_bytes, pl->need_sarr);
        pl->count_ns = 2;
        if (pl->mode == kModeTwoPass && 2 * (pl->smem + kSmemPerBlockReserved) > (size_t)kSmemPerSM) {
            // two CTAs with two slots each do not fit: one CTA with three slots
            const size_t s3 = CountSmemT<3>::total(pl->slot_bytes, tw, pl->need_sarr);
            if (s3 <= (size_t)kSmemBudget) {
                pl->smem = s3;
                pl->count_ns = 3;
            }
        }
        pl->smem_b = compact_smem_bytes(tw, X, pl->slot_bytes_b);
        if (pl->mode == kModeFused) {  // one kernel holds either role
            pl->smem = std::max(pl->smem, pl->smem_b);
            pl->smem_b = 0;
        }
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// samples as a 2-D tensor: rows = (fill, calo, crystal), columns = samples.
static bool encode_tensor_map(CUtensorMap *m, const int16_t *samples, int64_t rows, int64_t n_samples, int boxw,
                              int X)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n_samples, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)n_samples * sizeof(int16_t)};
    cuuint32_t box[2] = {(cuuint32_t)boxw, (cuuint32_t)X};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<int16_t *>(samples), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Estimated count-pass time per sample of a two-pass plan, relative to a tile
// that loads no halo with two CTAs per SM: the columns each tile loads (tile,
// halos and box rounding) per tile sample, times the cost of one CTA per SM.
// The count kernel is bound by the bytes it keeps in flight; one CTA with
// three slots ran 1.4x slower per loaded byte than two CTAs with two slots
// each (full fill, post = 64: 0.377 ms at 448 samples with one CTA per SM).
constexpr double kOneCountCtaCost = 1.4;

static double count_cost(const Plan &pl)
{
    const double cols = (double)pl.nbox * pl.boxw / pl.tw;
    const bool two_ctas = 2 * (pl.smem + kSmemPerBlockReserved) <= (size_t)kSmemPerSM;
    return two_ctas ? cols : cols * kOneCountCtaCost;
}

static int make_plan(int n_calo, int n_xtal, int64_t n_samples, int n_fills, const daq_params *p, Plan *pl)
{
    if (!p || n_calo < 0 || n_fills < 0 || n_samples < 0 || n_xtal < 1) return DAQ_EINVAL;
    if (n_xtal > kMaxXtal) return DAQ_EUNSUPPORTED;
    if (p->pre < 0 || p->post < 0 || p->pre + p->post > 512 || p->ped_samples < 1) return DAQ_EINVAL;
    if (p->n_decim < 0 || p->n_decim > 2) return DAQ_EINVAL;
    if (p->grid < -6) return DAQ_EINVAL;
    if (p->lag_tiles < 0) return DAQ_EINVAL;
    if (p->calo_base < 0 || p->q_calos < 0 ||
        (int64_t)p->calo_base + n_calo > (p->q_calos > 0 ? (int64_t)p->q_calos : (int64_t)n_calo))
        return DAQ_EINVAL;
    // scan fields: trailing run < 2^30 samples, island count < 2^31
    if (n_samples > ((int64_t)1 << 30) || (int64_t)n_fills * n_calo * n_samples > ((int64_t)1 << 32))
        return DAQ_EUNSUPPORTED;
    pl->need_sarr = 0;
    for (int d = 0; d < p->n_decim; ++d) {
        if (p->decim[d] < 1) return DAQ_EINVAL;
        if (p->decim[d] % 8) pl->need_sarr = 1;
    }
    if (p->tile != 0 && p->tile != 128 && p->tile != 224 && p->tile != 384 && p->tile != 448 && p->tile != 960)
        return DAQ_EINVAL;
    pl->mode = p->grid >= 0    ? kModeTwoPass
               : p->grid == -3 ? kModePipelined
               : p->grid == -4 ? kModeFused
               : p->grid == -5 ? kModeStream
               : p->grid == -6 ? kModePark
                               : kModePlain;
    const int hl = (p->post + 1 + 7) & ~7, hr = (p->pre + 1 + 7) & ~7;
    const int limit = p->tile ? p->tile : 448;
    // An explicit tile: the widest supported width not above it that fits.
    // Two-pass form with tile 0: the width of least estimated count-pass cost
    // (the slowest to fit wide halos).
    const bool by_cost = p->tile == 0 && pl->mode == kModeTwoPass;
    int chosen = -1;
    double best = 0.0;
    for (int tw : {960, 448, 384, 224, 128}) {
        if (tw > limit) continue;
        if (tw == 960 && pl->mode != kModePlain) continue;
        if (tw == 384 && pl->mode != kModeTwoPass) continue;
        if (tw + hl + hr > kMaxExtBits) continue;
        plan_geometry(pl, tw, p->pre, p->post, n_xtal);
        if (pl->smem > (size_t)kSmemBudget || pl->smem_b > (size_t)kSmemBudget) continue;
        if (!by_cost) {
            chosen = tw;
            break;
        }
        const double cost = count_cost(*pl);
        if (chosen < 0 || cost < best) {
            chosen = tw;
            best = cost;
        }
    }
    if (pl->mode == kModeTwoPass) {
        // The count pass normally loads each tile with its halo.  Where the
        // halo forces a narrower tile than allowed, or one count CTA per SM, it
        // loads the tile proper only (at the widest width) and the scan
        // completes the marks from the neighbouring tiles' crossings: at the
        // nominal windows both take the same count time and the completion
        // costs the scan a few microseconds; with post = 64 the halo-free pass
        // keeps 448-sample tiles with two count CTAs per SM.
        int widest = -1;
        for (int tw : {448, 384, 224, 128})
            if (tw <= limit) {
                widest = tw;
                break;
            }
        if (widest > 0) {
            if (chosen > 0 && chosen != pl->tw) plan_geometry(pl, chosen, p->pre, p->post, n_xtal);
            if (chosen < 0 || chosen < widest || pl->count_ns == 3) {
                chosen = widest;
                plan_geometry(pl, chosen, p->pre, p->post, n_xtal, true);
            }
        }
    }
    if (chosen < 0) return DAQ_EUNSUPPORTED;
    if (chosen != pl->tw) plan_geometry(pl, chosen, p->pre, p->post, n_xtal);
    pl->max_tiles = (int64_t)n_fills * n_calo * ((n_samples + chosen - 1) / chosen);
    pl->ws_tiles = pl->max_tiles;
    if (pl->mode == kModeStream || pl->mode == kModePark) {
        // these forms fall back to the two-pass form at run time when the rows
        // cannot be bulk-copied (or n_xtal is odd): its tiles may be narrower
        daq_params q = *p;
        q.grid = 0;
        Plan fb;
        if (make_plan(n_calo, n_xtal, n_samples, n_fills, &q, &fb) == DAQ_OK)
            pl->ws_tiles = std::max(pl->ws_tiles, fb.max_tiles);
    }
    return DAQ_OK;
}

template <typename K> static cudaError_t ensure_smem(K kernel, size_t bytes, size_t *configured)
{
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    if (dev >= 0 && dev < 64 && configured[dev] < bytes) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        configured[dev] = bytes;
    }
    return cudaSuccess;
}

template <int TW> static cudaError_t launch_plain(const KArgs &a, const Plan &pl, int grid, cudaStream_t s)
{
    static size_t configured[64] = {0};
    cudaError_t e = ensure_smem(daq_tile_kernel<TW>, pl.smem, configured);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, daq_tile_kernel<TW>, kThreads, pl.smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        int dev = 0;
        cudaGetDevice(&dev);
        grid = per_sm * device_info(dev).sms;
    }
    daq_tile_kernel<TW><<<grid, kThreads, pl.smem, s>>>(a);
    return cudaGetLastError();
}

template <int TW> static cudaError_t launch_pipe(const KArgs &a, const Plan &pl, int grid, cudaStream_t s)
{
    static size_t configured[64] = {0};
    cudaError_t e = ensure_smem(daq_pipe_kernel<TW>, pl.smem, configured);
    if (e != cudaSuccess) return e;
    daq_pipe_kernel<TW><<<grid, kPipeThreads, pl.smem, s>>>(a);
    return cudaGetLastError();
}

// Launch with programmatic stream serialization: the kernel may be scheduled
// while the previous kernel of the stream drains; it waits for it in-kernel
// (pdl_wait) before reading its outputs.
template <typename K>
static cudaError_t launch_pdl(K kernel, int grid, int block, size_t smem, cudaStream_t s, const KArgs &a)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return cudaErrorUnknown;
    cfg.attrs = attr;
    cfg.numAttrs = cap == cudaStreamCaptureStatusNone ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

// The count kernel for NS slots, halo-free or not, grids from occupancy when
// grid <= 0.
template <int TW, int NS, bool HF>
static cudaError_t launch_count(const KArgs &a, const Plan &pl, int grid, int sms, int64_t tiles, cudaStream_t s)
{
    static size_t conf[64] = {0};
    cudaError_t e = ensure_smem(daq_count_kernel<TW, NS, HF>, pl.smem, conf);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {
        int per = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, daq_count_kernel<TW, NS, HF>, count_threads<NS>(), pl.smem);
        if (e != cudaSuccess) return e;
        if (per < 1) return cudaErrorInvalidConfiguration;
        grid = per * sms;
    }
    grid = (int)std::min<int64_t>(grid, tiles);
    return launch_pdl(daq_count_kernel<TW, NS, HF>, grid, count_threads<NS>(), pl.smem, s, a);
}

// The compact kernel (DAQ_SPARSE: the form that passes over tiles without a
// marked sample), grids from occupancy when grid <= 0.
template <int TW, bool kSparse>
static cudaError_t launch_compact(const KArgs &a, const Plan &pl, int grid, int sms, int64_t tiles, cudaStream_t s)
{
    static size_t conf[64] = {0};
    cudaError_t e = ensure_smem(daq_compact_kernel<TW, kSparse>, pl.smem_b, conf);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {
        int per = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, daq_compact_kernel<TW, kSparse>, 256, pl.smem_b);
        if (e != cudaSuccess) return e;
        if (per < 1) return cudaErrorInvalidConfiguration;
        grid = per * sms;
    }
    grid = (int)std::min<int64_t>(grid, tiles);
    return launch_pdl(daq_compact_kernel<TW, kSparse>, grid, 256, pl.smem_b, s, a);
}

// Count pass, scan, compact pass.  Events (optional): [2] after the count
// kernel, [3] after the scan, [4] after the compact kernel.
template <int TW>
static cudaError_t launch_twopass(const KArgs &a, const Plan &pl, int grid, int sms, bool skip_isl,
                                  cudaEvent_t const *ev, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    const int64_t tiles = std::max<int64_t>(1, pl.max_tiles);
    e = pl.halo_free             ? launch_count<TW, 2, true>(a, pl, grid, sms, tiles, s)
        : pl.count_ns == 3       ? launch_count<TW, 3, false>(a, pl, grid, sms, tiles, s)
                                 : launch_count<TW, 2, false>(a, pl, grid, sms, tiles, s);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
    const int scan_blocks = (int)((tiles + kScanChunk - 1) / kScanChunk);
    e = pl.halo_free ? launch_pdl(daq_scan_kernel<TW, true>, scan_blocks, kScanThreads, 0, s, a)
                     : launch_pdl(daq_scan_kernel<TW, false>, scan_blocks, kScanThreads, 0, s, a);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
    if (!skip_isl) {
        e = (a.flags & DAQ_SPARSE) ? launch_compact<TW, true>(a, pl, grid, sms, tiles, s)
                                   : launch_compact<TW, false>(a, pl, grid, sms, tiles, s);
        if (e != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[4], s)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Streaming single-pass form: one persistent CTA per SM (at most one per tile).
template <int TW> static cudaError_t launch_stream(const KArgs &a, const Plan &pl, int sms, cudaStream_t s)
{
    static size_t conf[64] = {0};
    cudaError_t e = ensure_smem(daq_stream_kernel<TW>, pl.smem, conf);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, pl.max_tiles));
    daq_stream_kernel<TW><<<grid, kStrThreads, pl.smem, s>>>(a);
    return cudaGetLastError();
}

// Single-read form: one persistent CTA per SM (at most one per tile), launched
// with programmatic stream serialization behind the prepare kernel.
template <int TW> static cudaError_t launch_park(const KArgs &a, const Plan &pl, int sms, cudaStream_t s)
{
    static size_t conf[64] = {0};
    cudaError_t e = ensure_smem(daq_park_kernel<TW>, pl.smem, conf);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, pl.max_tiles));
    return launch_pdl(daq_park_kernel<TW>, grid, kPkThreads, pl.smem, s, a);
}

// Single-launch form: one cooperative launch of every CTA that fits (roles by
// block).  Events [2], [3] and [4] are all recorded after it.
template <int TW>
static cudaError_t launch_fused(const KArgs &a, const Plan &pl, int sms, cudaEvent_t const *ev, cudaStream_t s)
{
    static size_t conf[64] = {0};
    cudaError_t e = ensure_smem(daq_fused_kernel<TW>, pl.smem, conf);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, daq_fused_kernel<TW>, kCountThreads, pl.smem);
    if (e != cudaSuccess) return e;
    const int grid = per * sms;
    if (grid < 3) return cudaErrorInvalidConfiguration;
    void *args[] = {const_cast<KArgs *>(&a)};
    e = cudaLaunchCooperativeKernel((const void *)daq_fused_kernel<TW>, dim3(grid), dim3(kCountThreads), args,
                                    pl.smem, s);
    if (e != cudaSuccess) return e;
    for (int i = 2; i <= 4; ++i)
        if (ev && (e = cudaEventRecord(ev[i], s)) != cudaSuccess) return e;
    return cudaSuccess;
}

static int64_t q_bins(int64_t n, int32_t d) { return d > 0 ? (n + d - 1) / d : 0; }

// CUDA error behind this thread's last DAQ_ECUDA from daq_process_fills.
static thread_local cudaError_t t_last_cuda = cudaSuccess;
static int cuda_fail(cudaError_t e)
{
    t_last_cuda = e;
    return DAQ_ECUDA;
}

}  // namespace daq

using namespace daq;

extern "C" {

void daq_params_default(daq_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->threshold = 30;
    p->pre = 8;
    p->post = 24;
    p->ped_samples = 100;
    p->n_decim = 1;
    p->decim[0] = 32;
}

int64_t daq_q_bins(int64_t n_samples, int32_t decim) { return q_bins(n_samples, decim); }

int daq_workspace_size(int n_calo, int n_xtal, int64_t n_samples, int n_fills, const daq_params *params,
                       size_t *bytes)
{
    if (!bytes) return DAQ_EINVAL;
    Plan pl;
    const int rc = make_plan(n_calo, n_xtal, n_samples, n_fills, params, &pl);
    if (rc) return rc;
    *bytes = ws_layout(n_fills, n_calo, pl.ws_tiles).total;
    return DAQ_OK;
}

int daq_process_fills(const int16_t *samples, int n_calo, int n_xtal, int64_t n_samples, int n_fills,
                      const daq_params *params, const daq_islands *out, int64_t *qhist_inout)
{
    Plan pl;
    int rc = make_plan(n_calo, n_xtal, n_samples, n_fills, params, &pl);
    if (rc) return rc;
    const daq_params &p = *params;
    if (!out || !out->counts) return DAQ_EINVAL;
    const bool skip_isl = (p.flags & DAQ_SKIP_ISLANDS) != 0, skip_q = (p.flags & DAQ_SKIP_Q) != 0;
    const int64_t total = (int64_t)n_fills * n_calo * n_xtal * n_samples;
    if (total > 0 && !samples) return DAQ_EINVAL;
    if (!skip_isl) {
        if ((out->hdr_cap > 0 && !out->hdr) || (out->pool_row_cap > 0 && !out->pool) || out->hdr_cap < 0 ||
            out->pool_row_cap < 0)
            return DAQ_EINVAL;
        if ((reinterpret_cast<uintptr_t>(out->pool) & 15) || (reinterpret_cast<uintptr_t>(out->hdr) & 7))
            return DAQ_EINVAL;
    }
    const int64_t q_calos = p.q_calos > 0 ? p.q_calos : n_calo;
    int64_t q_total = 0;
    for (int d = 0; d < p.n_decim; ++d) q_total += q_bins(n_samples, p.decim[d]) * q_calos;
    if (!skip_q && q_total > 0 && !qhist_inout) return DAQ_EINVAL;
    if (reinterpret_cast<uintptr_t>(out->counts) & 7) return DAQ_EINVAL;
    const WsLayout wl = ws_layout(n_fills, n_calo, pl.ws_tiles);
    if (!p.workspace || p.workspace_bytes < wl.total || (reinterpret_cast<uintptr_t>(p.workspace) & 15))
        return DAQ_EINVAL;

    KArgs a;
    std::memset(&a, 0, sizeof(a));
    a.samples = samples;
    a.n_calo = n_calo;
    a.n_xtal = n_xtal;
    a.n_fills = n_fills;
    a.n_samples = n_samples;
    a.threshold = p.threshold;
    a.pre = p.pre;
    a.post = p.post;
    a.ped_samples = p.ped_samples;
    a.n_decim = p.n_decim;
    int64_t qoff = 0;
    for (int d = 0; d < p.n_decim; ++d) {
        a.decim[d] = p.decim[d];
        a.qbins[d] = q_bins(n_samples, p.decim[d]);
        a.qoff[d] = qoff;
        qoff += a.qbins[d] * q_calos;
    }
    a.fill_base = p.fill_base;
    a.calo_base = p.calo_base;
    a.q_calos = (int32_t)q_calos;
    a.wait_ns = p.wait_limit_ns ? p.wait_limit_ns : kWaitLimitNs;
    a.fill_len = p.fill_len;
    a.flags = p.flags;
    a.hl = pl.hl;
    a.hr = pl.hr;
    a.ew = pl.ew;
    a.rs = pl.rs;
    a.boxw = pl.boxw;
    a.nbox = pl.nbox;
    a.box_stride = pl.box_stride;
    a.slot_bytes = pl.slot_bytes;
    a.boxw_b = pl.boxw_b;
    a.nbox_b = pl.nbox_b;
    a.box_stride_b = pl.box_stride_b;
    a.slot_bytes_b = pl.slot_bytes_b;
    a.rs_b = pl.rs_b;
    a.mode = pl.mode;
    a.srow = stage_row_bytes(n_xtal);
    a.wpr = n_xtal / 2;
    a.wpr_mul = a.wpr > 0 ? (1ull << 32) / (unsigned long long)a.wpr + 1 : 0ull;
    a.use_tma = 0;
    if (total > 0 && n_samples % 8 == 0 && (reinterpret_cast<uintptr_t>(samples) & 15) == 0)
        a.use_tma = encode_tensor_map(&a.tmap, samples, (int64_t)n_fills * n_calo * n_xtal, n_samples, pl.boxw,
                                      n_xtal) &&
                    encode_tensor_map(&a.tmap_b, samples, (int64_t)n_fills * n_calo * n_xtal, n_samples,
                                      pl.boxw_b, n_xtal);
    if (pl.mode == kModeStream && a.use_tma) {
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        cuuint64_t dims[2] = {(cuuint64_t)n_samples, (cuuint64_t)((int64_t)n_fills * n_calo * n_xtal)};
        cuuint64_t strides[1] = {(cuuint64_t)n_samples * sizeof(int16_t)};
        cuuint32_t box[2] = {(cuuint32_t)kStrStep, (cuuint32_t)n_xtal};
        cuuint32_t estr[2] = {1, 1};
        a.use_tma = enc && enc(&a.tmap_c, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<int16_t *>(samples), dims,
                               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if ((pl.mode == kModeStream && !a.use_tma) || (pl.mode == kModePark && (!a.use_tma || (n_xtal & 1)))) {
        // the streaming form reads 16-byte groups and bulk-copies tiles, the
        // single-read form moves whole 32-bit words of pool rows: rows that
        // are not 16-byte aligned (or odd crystal counts) take the two-pass form
        daq_params q = p;
        q.grid = 0;
        rc = make_plan(n_calo, n_xtal, n_samples, n_fills, &q, &pl);
        if (rc) return rc;
        a.hl = pl.hl;
        a.hr = pl.hr;
        a.ew = pl.ew;
        a.rs = pl.rs;
        a.boxw = pl.boxw;
        a.nbox = pl.nbox;
        a.box_stride = pl.box_stride;
        a.slot_bytes = pl.slot_bytes;
        a.boxw_b = pl.boxw_b;
        a.nbox_b = pl.nbox_b;
        a.box_stride_b = pl.box_stride_b;
        a.slot_bytes_b = pl.slot_bytes_b;
        a.rs_b = pl.rs_b;
        a.mode = pl.mode;
        if (total > 0 && n_samples % 8 == 0 && (reinterpret_cast<uintptr_t>(samples) & 15) == 0)
            a.use_tma = encode_tensor_map(&a.tmap, samples, (int64_t)n_fills * n_calo * n_xtal, n_samples, pl.boxw,
                                          n_xtal) &&
                        encode_tensor_map(&a.tmap_b, samples, (int64_t)n_fills * n_calo * n_xtal, n_samples,
                                          pl.boxw_b, n_xtal);
    }
    a.need_sarr = pl.need_sarr;
    a.halo_free = pl.halo_free;
    a.max_tiles = pl.max_tiles;
    a.lag_tiles = std::max<int64_t>(p.lag_tiles > 0 ? p.lag_tiles : kFusedLagTiles, kFusedMinLag);
    a.str_meta = pl.str_meta;
    a.str_stages = pl.str_stages;
    a.pk_slots = pl.pk_slots;
    a.pk_cols = pl.pk_cols;
    a.hdr = skip_isl ? nullptr : out->hdr;
    a.hdr_cap = skip_isl ? 0 : out->hdr_cap;
    a.pool = skip_isl ? nullptr : out->pool;
    a.pool_cap = skip_isl ? 0 : out->pool_row_cap;
    a.ped_out = out->pedestal;
    a.counts = out->counts;
    a.q = qhist_inout;
    unsigned char *ws = static_cast<unsigned char *>(p.workspace);
    a.ticket = reinterpret_cast<unsigned int *>(ws + wl.ticket);
    a.fctr = reinterpret_cast<unsigned long long *>(ws + 128);
    a.fill_tile_start = reinterpret_cast<long long *>(ws + wl.fts);
    a.lens = reinterpret_cast<int32_t *>(ws + wl.lens);
    a.ptot = reinterpret_cast<int32_t *>(ws + wl.ptot);
    a.status = reinterpret_cast<TileStatus *>(ws + wl.status);
    a.marks = reinterpret_cast<uint32_t *>(ws + wl.marks);
    a.recs = ws + wl.recs;
    a.excl = ws + wl.excl;
    a.scan_status = reinterpret_cast<TileStatus *>(ws + wl.scan_status);
    a.scan_ticket = reinterpret_cast<unsigned int *>(ws + 384);
    a.trace = reinterpret_cast<unsigned long long *>(p.trace);

    cudaStream_t s = static_cast<cudaStream_t>(p.stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DAQ_ECUDA;
    const DeviceInfo di = device_info(dev);
    if (di.sms <= 0) return DAQ_ECUDA;
    if ((int)pl.smem > di.smem_optin || (int)pl.smem_b > di.smem_optin) return DAQ_EUNSUPPORTED;

    cudaEvent_t const *ev = reinterpret_cast<cudaEvent_t const *>(p.events);
    if (ev && cudaEventRecord(ev[0], s) != cudaSuccess) return DAQ_ECUDA;
    const long long n_cf = (long long)n_fills * n_calo;
    const int prep_grid = (int)std::max<long long>(1, std::min<long long>(std::max<long long>(n_cf, 1), 4ll * di.sms));
    daq_prepare_kernel<<<prep_grid, kThreads, 0, s>>>(a, pl.tw);
    if (cudaError_t e0 = cudaGetLastError()) return cuda_fail(e0);
    if (ev && cudaEventRecord(ev[1], s) != cudaSuccess) return DAQ_ECUDA;

    const int64_t tiles_cap = std::max<int64_t>(1, std::min<int64_t>(pl.max_tiles, INT32_MAX));
    cudaError_t e;
    if (pl.mode == kModePark) {
        switch (pl.tw) {
        case 128: e = launch_park<128>(a, pl, di.sms, s); break;
        case 224: e = launch_park<224>(a, pl, di.sms, s); break;
        default: e = launch_park<448>(a, pl, di.sms, s); break;
        }
    } else if (pl.mode == kModeStream) {
        switch (pl.tw) {
        case 128: e = launch_stream<128>(a, pl, di.sms, s); break;
        case 224: e = launch_stream<224>(a, pl, di.sms, s); break;
        default: e = launch_stream<448>(a, pl, di.sms, s); break;
        }
    } else if (pl.mode == kModeFused) {
        switch (pl.tw) {
        case 128: e = launch_fused<128>(a, pl, di.sms, ev, s); break;
        case 224: e = launch_fused<224>(a, pl, di.sms, ev, s); break;
        default: e = launch_fused<448>(a, pl, di.sms, ev, s); break;
        }
    } else if (pl.mode == kModeTwoPass) {
        switch (pl.tw) {
        case 128: e = launch_twopass<128>(a, pl, p.grid, di.sms, skip_isl, ev, s); break;
        case 224: e = launch_twopass<224>(a, pl, p.grid, di.sms, skip_isl, ev, s); break;
        case 384: e = launch_twopass<384>(a, pl, p.grid, di.sms, skip_isl, ev, s); break;
        default: e = launch_twopass<448>(a, pl, p.grid, di.sms, skip_isl, ev, s); break;
        }
    } else if (pl.mode == kModePipelined) {
        int grid = p.grid > 0 ? p.grid : di.sms;
        grid = (int)std::min<int64_t>(grid, tiles_cap);
        switch (pl.tw) {
        case 128: e = launch_pipe<128>(a, pl, grid, s); break;
        case 224: e = launch_pipe<224>(a, pl, grid, s); break;
        case 448: e = launch_pipe<448>(a, pl, grid, s); break;
        default: e = launch_pipe<960>(a, pl, grid, s); break;
        }
    } else {
        const int grid = p.grid == -1 ? (int)tiles_cap : 0;  // -1: one CTA per tile; -2: persistent
        switch (pl.tw) {
        case 128: e = launch_plain<128>(a, pl, grid, s); break;
        case 224: e = launch_plain<224>(a, pl, grid, s); break;
        case 448: e = launch_plain<448>(a, pl, grid, s); break;
        default: e = launch_plain<960>(a, pl, grid, s); break;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (ev && pl.mode != kModeTwoPass)
        for (int k = 2; k < 5; ++k)
            if (cudaEventRecord(ev[k], s) != cudaSuccess) return DAQ_ECUDA;

    if (p.flags & DAQ_SYNC) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return DAQ_ECUDA;
        int64_t h[4];
        if (cudaMemcpy(h, out->counts, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return DAQ_ECUDA;
        return daq_status_from_counts(h);
    }
    return DAQ_OK;
}

int64_t daq_trace_tiles(int n_calo, int n_xtal, int64_t n_samples, int n_fills, const daq_params *params)
{
    Plan pl;
    if (make_plan(n_calo, n_xtal, n_samples, n_fills, params, &pl) != DAQ_OK) return 0;
    return pl.ws_tiles;
}

int daq_status_from_counts(const int64_t *c)
{
    if (!c) return DAQ_EINVAL;
    if (c[2] & DAQ_DEV_TIMEOUT) return DAQ_ETIMEOUT;
    if (c[2] & DAQ_DEV_BAD_FILL_LEN) return DAQ_EINVAL;
    if (c[2] & DAQ_DEV_BAD_INDEX) return DAQ_EINDEX;
    if (c[2] & (DAQ_DEV_HDR_OVERFLOW | DAQ_DEV_POOL_OVERFLOW)) return DAQ_ECAPACITY;
    return DAQ_OK;
}

const char *daq_strerror(int status)
{
    switch (status) {
    case DAQ_OK: return "success";
    case DAQ_EINVAL: return "invalid argument (shape, parameter, pointer, alignment or workspace size)";
    case DAQ_ECAPACITY: return "island records or pool rows exceeded their capacity; counts hold the sizes needed";
    case DAQ_ECUDA: return "CUDA call or kernel launch failed";
    case DAQ_ETIMEOUT: return "a bounded device-side wait gave up; outputs are incomplete";
    case DAQ_EUNSUPPORTED: return "request not supported by this build";
    case DAQ_ESCRATCH: return "the call needs more scratch than the library's built-in area holds";
    case DAQ_EINDEX: return "a device-side index check (DAQ_DEBUG_CHECKS) failed; the store was skipped";
    default: return "unknown status";
    }
}

int daq_version(void) { return 102; }

const char *daq_last_cuda_error(void)
{
    static thread_local char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", cudaGetErrorName(t_last_cuda), cudaGetErrorString(t_last_cuda));
    return buf;
}

}  // extern "C"
