// Fused per-fill processing of muon g-2 calorimeter waveforms on sm_103a.
//
// Paper: W. Gohn, arXiv:1611.04959, Sec. 3 and Table 2.  The eight kernels of
// Table 2 (pedestal, threshold, pre/post samples, merge, save islands, sum,
// Q decimation, fill-by-fill sum) become two launches:
//
//   daq_prepare_kernel  pedestals (Table 2 row 1) for every (fill, calo,
//                       crystal), the per-fill tile plan, and the reset of the
//                       scan workspace;
//   daq_tile_kernel     one pass over the samples.  A persistent CTA takes
//                       tiles of TW samples of one calorimeter-fill in order
//                       (atomic ticket), bulk-copies the 54 crystal rows of the
//                       tile plus a halo into shared memory, and from there:
//                       sums crystals and subtracts pedestals (row 6), tests
//                       the threshold (row 2), widens crossings by the pre/post
//                       windows (row 3), finds island starts and ends (row 4),
//                       takes its global pool-row and island offsets from a
//                       single-pass decoupled look-back scan over tiles, writes
//                       island records and time-major pool rows (row 5), and
//                       adds decimated partial sums into the int64 Q
//                       histograms (rows 7-8).
//
// Every quantity is an integer, so the result does not depend on tile size,
// grid size or the order in which tiles run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "daq.h"
#include "daq_device.cuh"

namespace daq {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxXtal = 64;
constexpr int kMaxExtBits = 1024;            // tile + halos, one warp of 32-bit words
constexpr uint64_t kWaitLimitNs = 4000000000ull;  // bounded device waits (4 s)

// Scan state of one tile: aggregate and inclusive prefix, each a (flag, payload) pair.
// flag word  = (marked samples << 2) | kind, kind 1 = valid, 2 = poisoned
// payload    = (island starts << 32) | (trailing run << 1) | continues
struct TileStatus {
    unsigned long long agg_payload, agg_flag;
    unsigned long long inc_payload, inc_flag;
};

struct Agg {
    long long m;   // marked samples (pool rows)
    long long s;   // island starts
    long long tr;  // marked samples in the run that ends at the last sample
    int full;      // every sample marked and the run continues from the previous tile
    int poison;
};

__device__ __forceinline__ Agg agg_identity() { return Agg{0, 0, 0, 1, 0}; }

// Prefix p followed by tile t.
__device__ __forceinline__ Agg combine(const Agg &p, const Agg &t)
{
    Agg r;
    r.m = p.m + t.m;
    r.s = p.s + t.s;
    r.tr = t.full ? p.tr + t.tr : t.tr;
    r.full = p.full && t.full;
    r.poison = p.poison | t.poison;
    return r;
}

__device__ __forceinline__ void agg_encode(const Agg &a, unsigned long long &flag, unsigned long long &payload)
{
    flag = ((unsigned long long)a.m << 2) | (a.poison ? 2ull : 1ull);
    payload = ((unsigned long long)a.s << 32) | ((unsigned long long)a.tr << 1) | (unsigned long long)(a.full != 0);
}

__device__ __forceinline__ Agg agg_decode(unsigned long long flag, unsigned long long payload)
{
    Agg a;
    a.m = (long long)(flag >> 2);
    a.poison = (flag & 3ull) == 2ull;
    a.s = (long long)(payload >> 32);
    a.tr = (long long)((payload >> 1) & 0x7fffffffull);
    a.full = (int)(payload & 1ull);
    return a;
}

__device__ __forceinline__ Agg shfl_agg(const Agg &a, int src)
{
    Agg r;
    r.m = __shfl_sync(kFull, a.m, src);
    r.s = __shfl_sync(kFull, a.s, src);
    r.tr = __shfl_sync(kFull, a.tr, src);
    r.full = __shfl_sync(kFull, a.full, src);
    r.poison = __shfl_sync(kFull, a.poison, src);
    return r;
}

struct KArgs {
    const int16_t *samples;
    int32_t n_calo, n_xtal, n_fills;
    int64_t n_samples;  // row pitch
    int32_t threshold, pre, post, ped_samples;
    int32_t n_decim, decim[2];
    int64_t qbins[2], qoff[2];
    int32_t fill_base;
    const int32_t *fill_len;
    uint32_t flags;
    int32_t hl, hr, ew, rs;  // halo left/right, extended width, smem row stride (bytes)
    int32_t bulk_ok;
    int32_t need_sarr;
    int64_t max_tiles;
    // outputs
    daq_island *hdr;
    int64_t hdr_cap;
    int16_t *pool;
    int64_t pool_cap;
    int32_t *ped_out;
    int64_t *counts;
    int64_t *q;
    // workspace
    unsigned int *ticket;
    long long *fill_tile_start;  // [n_fills + 1]
    int32_t *lens;               // [n_fills], clamped
    int32_t *ptot;               // [n_fills * n_calo]
    TileStatus *status;          // [max_tiles]
};

// Workspace layout (byte offsets from the workspace base).
struct WsLayout {
    size_t ticket, fts, lens, ptot, status, total;
};

static WsLayout ws_layout(int64_t n_fills, int64_t n_calo, int64_t max_tiles)
{
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    WsLayout w;
    w.ticket = 0;
    w.fts = up(16);
    w.lens = up(w.fts + sizeof(long long) * (size_t)(n_fills + 1));
    w.ptot = up(w.lens + sizeof(int32_t) * (size_t)(n_fills > 0 ? n_fills : 1));
    w.status = up(w.ptot + sizeof(int32_t) * (size_t)(n_fills * n_calo > 0 ? n_fills * n_calo : 1));
    w.total = up(w.status + sizeof(TileStatus) * (size_t)(max_tiles > 0 ? max_tiles : 1));
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
// tile-status array and the ticket.
__global__ void __launch_bounds__(kThreads) daq_prepare_kernel(KArgs a, int tw)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ long long s_warp[kWarps];
    __shared__ long long s_carry;

    // reset of the scan state
    {
        uint4 *st = reinterpret_cast<uint4 *>(a.status);
        const long long n16 = a.max_tiles * (long long)(sizeof(TileStatus) / 16);
        for (long long i = (long long)blockIdx.x * kThreads + tid; i < n16; i += (long long)gridDim.x * kThreads)
            st[i] = make_uint4(0u, 0u, 0u, 0u);
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
            long long ex = warp_excl_scan_add<long long>(tiles, lane, tot);
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
        if (__syncthreads_or(bad) && tid == 0)
            atomicOr(reinterpret_cast<unsigned long long *>(&a.counts[2]), (unsigned long long)DAQ_DEV_BAD_FILL_LEN);
    }

    // pedestals: warp per crystal, block per calorimeter-fill
    __shared__ long long s_ped[kWarps];
    const long long n_cf = (long long)a.n_fills * a.n_calo;
    for (long long cf = blockIdx.x; cf < n_cf; cf += gridDim.x) {
        const int f = (int)(cf / a.n_calo);
        long long len = a.fill_len ? (long long)a.fill_len[f] : a.n_samples;
        len = len < 0 ? 0 : (len > a.n_samples ? a.n_samples : len);
        const long long n = len < a.ped_samples ? len : a.ped_samples;
        long long ptot_part = 0;
        for (int x = warp; x < a.n_xtal; x += kWarps) {
            const int16_t *row = a.samples + (cf * a.n_xtal + x) * a.n_samples;
            long long sum = 0;
            for (long long t = lane; t < n; t += 32) sum += row[t];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(kFull, sum, d);
            const long long p = n > 0 ? floor_div_ll(sum + n / 2, n) : 0;
            if (lane == 0 && a.ped_out && !(a.flags & DAQ_SKIP_ISLANDS)) a.ped_out[cf * a.n_xtal + x] = (int32_t)p;
            ptot_part += p;
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

// ============================================================================ tile kernel
struct TileCtrl {
    long long tile;
    long long t0, len, t_end;
    int f, c, ptot, bail;
    Agg agg, excl;
};

template <int TW>
__global__ void __launch_bounds__(kThreads, 2) daq_tile_kernel(KArgs a)
{
    constexpr int NWT = TW / 32;  // bit words of the tile proper
    constexpr int NBT = TW / 8;   // 8-sample blocks of the tile proper
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int X = a.n_xtal, RS = a.rs, HL = a.hl, EW = a.ew;
    const int NB = EW / 8;               // 8-sample blocks incl. halos
    const int NWE = (EW + 31) / 32;      // bit words incl. halos

    // ---- shared memory carve-up
    unsigned char *tbuf = smem;                                   // X rows x RS bytes
    unsigned char *zrow = tbuf + (size_t)X * RS;                  // one zero row
    unsigned char *stage = zrow + RS;                             // TW * 2X + 32 bytes
    const int stage_bytes = ((TW * 2 * X + 32) + 15) & ~15;
    uint8_t *abyte = stage + stage_bytes;                         // 128 bytes of threshold bits
    int32_t *blocksum = reinterpret_cast<int32_t *>(abyte + 128); // NBT
    int32_t *sarr = blocksum + NBT;                               // TW (only when a decimation % 8 != 0)
    uint32_t *w_m = reinterpret_cast<uint32_t *>(sarr + (a.need_sarr ? TW : 0));
    uint32_t *w_s = w_m + NWT;
    uint32_t *w_e = w_s + NWT;
    int32_t *w_mb = reinterpret_cast<int32_t *>(w_e + NWT);       // marked before word
    int32_t *w_sb = w_mb + NWT;                                   // starts before word
    int32_t *w_ls = w_sb + NWT;                                   // last start before word (tile-relative), -1
    TileCtrl *ctrl = reinterpret_cast<TileCtrl *>((reinterpret_cast<uintptr_t>(w_ls + NWT) + 15) & ~uintptr_t(15));
    uint64_t *bar = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(ctrl + 1) + 15) & ~uintptr_t(15));

    // ---- one-time setup
    for (int i = tid; i < RS / 4; i += kThreads) reinterpret_cast<uint32_t *>(zrow)[i] = 0u;
    for (int i = tid; i < 32; i += kThreads) reinterpret_cast<uint32_t *>(abyte)[i] = 0u;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    // ldmatrix row addresses: lane L feeds crystal L (first x4) and 32 + L (second x4);
    // rows past n_xtal read the zero row
    const uint32_t tile_s = smem_addr(tbuf), zrow_s = smem_addr(zrow);
    const uint32_t a_lo = lane < X ? tile_s + (uint32_t)(lane * RS) : zrow_s;
    const uint32_t a_hi = lane + 32 < X ? tile_s + (uint32_t)((lane + 32) * RS) : zrow_s;
    const bool two_groups = X > 32;

    uint32_t phase = 0;
    for (;;) {
        // ------------------------------------------------------------ ticket + decode
        if (tid == 0) {
            TileCtrl &C = *ctrl;
            const long long total = a.fill_tile_start[a.n_fills];
            const long long tile = (long long)atomicAdd(a.ticket, 1u);
            C.tile = tile;
            C.bail = 0;
            if (tile < total) {
                int lo = 0, hi = a.n_fills - 1;  // last fill with start <= tile
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.fill_tile_start[mid] <= tile) lo = mid; else hi = mid - 1;
                }
                const long long len = a.lens[lo];
                const long long tpc = (len + TW - 1) / TW;
                const long long rem = tile - a.fill_tile_start[lo];
                C.f = lo;
                C.c = (int)(rem / tpc);
                C.t0 = (rem % tpc) * TW;
                C.len = len;
                C.t_end = min(C.t0 + TW, len);
                C.ptot = a.ptot[(long long)lo * a.n_calo + C.c];
            }
        }
        __syncthreads();
        const long long tile = ctrl->tile;
        if (tile >= a.fill_tile_start[a.n_fills]) break;
        const int f = ctrl->f, c = ctrl->c, ptot = ctrl->ptot;
        const long long t0 = ctrl->t0, len = ctrl->len, t_end = ctrl->t_end;
        const long long cf = (long long)f * a.n_calo + c;
        const int16_t *rows = a.samples + cf * X * a.n_samples;
        const long long e0 = t0 - HL;  // sample of extended column 0

        // ------------------------------------------------------------ load tile + halo
        if (a.bulk_ok) {
            const long long lo = max(e0, 0ll);
            const long long hi = min((long long)(t0 + TW + a.hr), (long long)a.n_samples);
            const uint32_t row_bytes = (uint32_t)((hi - lo) * 2);
            if (warp == 0) {
                fence_proxy_async_smem();
                if (lane == 0) mbar_arrive_expect_tx(bar, row_bytes * (uint32_t)X);
                __syncwarp();
                for (int x = lane; x < X; x += 32)
                    bulk_g2s(tbuf + (size_t)x * RS + (lo - e0) * 2, rows + (long long)x * a.n_samples + lo, row_bytes,
                             bar);
            }
            const bool ok = mbar_wait_bounded(bar, phase, kWaitLimitNs);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicOr(reinterpret_cast<unsigned long long *>(&a.counts[2]),
                                       (unsigned long long)DAQ_DEV_TIMEOUT);
                mbar_wait_bounded(bar, phase ^ 1u, kWaitLimitNs);
                return;
            }
        } else {
            for (int i = tid; i < X * EW; i += kThreads) {
                const int x = i / EW, col = i - x * EW;
                const long long t = e0 + col;
                int16_t v = 0;
                if (t >= 0 && t < a.n_samples) v = rows[(long long)x * a.n_samples + t];
                reinterpret_cast<int16_t *>(tbuf + (size_t)x * RS)[col] = v;
            }
            __syncthreads();
        }

        // ------------------------------------------------------------ sums, threshold bits, block sums
        for (int b = warp; b < NB; b += kWarps) {
            const uint32_t col = 16u * (uint32_t)b;
            uint32_t r0, r1, r2, r3, r4 = 0, r5 = 0, r6 = 0, r7 = 0;
            ldsm_x4_trans(a_lo + col, r0, r1, r2, r3);
            if (two_groups) ldsm_x4_trans(a_hi + col, r4, r5, r6, r7);
            int acc = __dp2a_lo((int)r0, 0x0101, 0);
            acc = __dp2a_lo((int)r1, 0x0101, acc);
            acc = __dp2a_lo((int)r2, 0x0101, acc);
            acc = __dp2a_lo((int)r3, 0x0101, acc);
            acc = __dp2a_lo((int)r4, 0x0101, acc);
            acc = __dp2a_lo((int)r5, 0x0101, acc);
            acc = __dp2a_lo((int)r6, 0x0101, acc);
            acc = __dp2a_lo((int)r7, 0x0101, acc);
            acc += __shfl_xor_sync(kFull, acc, 1);
            acc += __shfl_xor_sync(kFull, acc, 2);
            const int j = lane >> 2;
            const long long t = e0 + 8 * b + j;
            const int S = acc - ptot;
            const bool cross = (t >= 0) && (t < len) && (S > a.threshold);
            uint32_t v = __ballot_sync(kFull, cross) & 0x11111111u;
            v = (v | (v >> 3)) & 0x03030303u;
            v = (v | (v >> 6)) & 0x000f000fu;
            v = (v | (v >> 12)) & 0xffu;
            if (lane == 0) abyte[b] = (uint8_t)v;
            const int bt = b - HL / 8;
            if (bt >= 0 && bt < NBT) {
                const bool in = t < t_end;
                int sv = in ? S : 0;
                sv += __shfl_xor_sync(kFull, sv, 4);
                sv += __shfl_xor_sync(kFull, sv, 8);
                sv += __shfl_xor_sync(kFull, sv, 16);
                if (lane == 0) blocksum[bt] = sv;
                if (a.need_sarr && (lane & 3) == 0 && in) sarr[8 * bt + j] = S;
            }
        }
        __syncthreads();

        if (warp == 0) {
            // -------------------------------------------------------- windows, merge, tile aggregate
            const uint32_t A = lane < NWE ? reinterpret_cast<const uint32_t *>(abyte)[lane] : 0u;
            // forward spread: F[i] = OR_{k=0..post} A[i-k]
            uint32_t Fv = A;
            int cov = 1;
            while (2 * cov <= a.post + 1) {
                Fv |= shl_bits(Fv, cov, lane);
                cov *= 2;
            }
            if (cov < a.post + 1) Fv |= shl_bits(Fv, a.post + 1 - cov, lane);
            // backward spread: M[i] = OR_{k=0..pre} F[i+k]
            uint32_t Mv = Fv;
            cov = 1;
            while (2 * cov <= a.pre + 1) {
                Mv |= shr_bits(Mv, cov, lane);
                cov *= 2;
            }
            if (cov < a.pre + 1) Mv |= shr_bits(Mv, a.pre + 1 - cov, lane);
            // samples outside [0, len) are never marked
            Mv &= range_mask(32ll * lane, -e0, len - e0);
            // marks of t0 - 1 and t0 + TW (extended bits HL - 1 and HL + TW)
            const uint32_t m_prev = (__shfl_sync(kFull, Mv, (HL - 1) >> 5) >> ((HL - 1) & 31)) & 1u;
            const uint32_t m_next = (__shfl_sync(kFull, Mv, (HL + TW) >> 5) >> ((HL + TW) & 31)) & 1u;
            // tile-relative words: bits [HL + 32w, HL + 32w + 32)
            const int qo = HL >> 5, sh = HL & 31;
            uint32_t lo_w = __shfl_down_sync(kFull, Mv, qo);
            uint32_t hi_w = __shfl_down_sync(kFull, Mv, min(qo + 1, 31));
            if (lane + qo > 31) lo_w = 0u;
            if (lane + qo + 1 > 31) hi_w = 0u;
            uint32_t Mt = sh ? ((lo_w >> sh) | (hi_w << (32 - sh))) : lo_w;
            if (lane >= NWT) Mt = 0u;
            uint32_t below = __shfl_up_sync(kFull, Mt, 1);
            if (lane == 0) below = m_prev << 31;
            uint32_t above = __shfl_down_sync(kFull, Mt, 1);
            if (lane == NWT - 1) above = m_next;
            if (lane >= NWT) above = 0u;
            const uint32_t St = Mt & ~((Mt << 1) | (below >> 31));
            const uint32_t Et = Mt & ~((Mt >> 1) | (above << 31));
            int m_tot, s_tot;
            const int mb = warp_excl_scan_add<int>(__popc(Mt), lane, m_tot);
            const int sb = warp_excl_scan_add<int>(__popc(St), lane, s_tot);
            const int last_start = St ? 32 * lane + 31 - __clz(St) : -1;
            const int ls = warp_excl_scan_max(last_start, lane, -1);
            const int nt = (int)(t_end - t0);
            const uint32_t zeros = ~Mt & range_mask(32ll * lane, 0, nt);
            const int lz = warp_max(zeros ? 32 * lane + 31 - __clz(zeros) : -1);
            if (lane < NWT) {
                w_m[lane] = Mt;
                w_s[lane] = St;
                w_e[lane] = Et;
                w_mb[lane] = mb;
                w_sb[lane] = sb;
                w_ls[lane] = ls;
            }
            Agg agg;
            agg.m = m_tot;
            agg.s = s_tot;
            agg.tr = nt - 1 - lz;
            agg.full = (lz < 0) && m_prev;
            agg.poison = 0;
            __syncwarp();
            // let the other warps start writing the staged rows
            asm volatile("bar.arrive 1, %0;" ::"r"(kThreads) : "memory");

            // -------------------------------------------------------- decoupled look-back
            TileStatus *st = a.status;
            Agg excl = agg_identity();
            if (tile == 0) {
                if (lane == 0) {
                    unsigned long long fl, pl;
                    agg_encode(agg, fl, pl);
                    st_relaxed_u64(&st[0].inc_payload, pl);
                    st_release_u64(&st[0].inc_flag, fl);
                }
            } else {
                if (lane == 0) {
                    unsigned long long fl, pl;
                    agg_encode(agg, fl, pl);
                    st_relaxed_u64(&st[tile].agg_payload, pl);
                    st_release_u64(&st[tile].agg_flag, fl);
                }
                long long pos = tile - 1;
                Agg acc = agg_identity();
                const uint64_t tstart = global_ns();
                bool timed_out = false;
                for (uint32_t iter = 0;; ++iter) {
                    const long long idx = pos - lane;
                    int kind = 2;
                    Agg v = agg_identity();
                    if (idx >= 0) {
                        kind = 0;
                        unsigned long long fl = ld_acquire_u64(&st[idx].inc_flag);
                        if (fl & 3ull) {
                            kind = 2;
                            v = agg_decode(fl, ld_relaxed_u64(&st[idx].inc_payload));
                        } else {
                            fl = ld_acquire_u64(&st[idx].agg_flag);
                            if (fl & 3ull) {
                                kind = 1;
                                v = agg_decode(fl, ld_relaxed_u64(&st[idx].agg_payload));
                            }
                        }
                    }
                    const uint32_t incm = __ballot_sync(kFull, kind == 2);
                    const uint32_t ready = __ballot_sync(kFull, kind != 0);
                    const int stop = incm ? __ffs(incm) - 1 : 31;
                    const uint32_t need = stop == 31 ? kFull : ((2u << stop) - 1u);
                    if ((ready & need) == need) {
                        Agg w = shfl_agg(v, stop);
                        for (int i = stop - 1; i >= 0; --i) w = combine(w, shfl_agg(v, i));
                        acc = combine(w, acc);
                        if (incm) break;
                        pos -= 32;
                        continue;
                    }
                    if ((iter & 31u) == 31u) {
                        bool give_up = global_ns() - tstart > kWaitLimitNs;
                        if (lane == 0 && (ld_relaxed_u64(reinterpret_cast<const unsigned long long *>(&a.counts[2])) &
                                          DAQ_DEV_TIMEOUT))
                            give_up = true;
                        if (__shfl_sync(kFull, (int)give_up, 0)) {
                            timed_out = true;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                excl = acc;
                if (timed_out) {
                    excl.poison = 1;
                    if (lane == 0)
                        atomicOr(reinterpret_cast<unsigned long long *>(&a.counts[2]),
                                 (unsigned long long)DAQ_DEV_TIMEOUT);
                }
                if (lane == 0) {
                    unsigned long long fl, pl;
                    agg_encode(combine(excl, agg), fl, pl);
                    st_relaxed_u64(&st[tile].inc_payload, pl);
                    st_release_u64(&st[tile].inc_flag, fl);
                }
            }
            if (lane == 0) {
                ctrl->agg = agg;
                ctrl->excl = excl;
            }
        } else {
            // -------------------------------------------------------- Q: decimate + fill-by-fill sum
            if (!(a.flags & DAQ_SKIP_Q)) {
                for (int d = 0; d < a.n_decim; ++d) {
                    const long long D = a.decim[d];
                    unsigned long long *qrow =
                        reinterpret_cast<unsigned long long *>(a.q + a.qoff[d] + (long long)c * a.qbins[d]);
                    const long long k_lo = t0 / D, k_hi = (t_end - 1) / D;
                    for (long long k = k_lo + (tid - 32); k <= k_hi; k += kThreads - 32) {
                        const long long lo = max(k * D, t0) - t0, hi = min(k * D + D, t_end) - t0;
                        long long sum = 0;
                        if ((D & 7) == 0) {
                            for (long long b = lo >> 3; b < (hi + 7) >> 3; ++b) sum += blocksum[b];
                        } else {
                            for (long long t = lo; t < hi; ++t) sum += sarr[t];
                        }
                        atomicAdd(qrow + k, (unsigned long long)sum);
                    }
                }
            }
            // -------------------------------------------------------- stage pool rows (tile-local order)
            asm volatile("bar.sync 1, %0;" ::"r"(kThreads) : "memory");
            if (!(a.flags & DAQ_SKIP_ISLANDS)) {
                const int q4 = lane & 3, j = lane >> 2;
                const int row_bytes = 2 * X;
                for (int bt = warp - 1; bt < NBT; bt += kWarps - 1) {
                    const int w = bt >> 2, shift = (bt & 3) * 8;
                    const uint32_t mw = w_m[w];
                    const uint32_t bits = (mw >> shift) & 0xffu;
                    if (!bits) continue;
                    const uint32_t col = 16u * (uint32_t)(bt + HL / 8);
                    uint32_t r[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
                    ldsm_x4_trans(a_lo + col, r[0], r[1], r[2], r[3]);
                    if (two_groups) ldsm_x4_trans(a_hi + col, r[4], r[5], r[6], r[7]);
                    if (!((bits >> j) & 1u)) continue;
                    const int bitpos = shift + j;
                    const int rl = w_mb[w] + __popc(mw & ((1u << bitpos) - 1u));
                    unsigned char *dst = stage + (size_t)rl * row_bytes;
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        if (g >= 4 && !two_groups) break;
                        const int x = 8 * g + 2 * q4;
                        if (x >= X) continue;
                        if (x + 1 < X && !(X & 1)) {
                            *reinterpret_cast<uint32_t *>(dst + 2 * x) = r[g];
                        } else {
                            *reinterpret_cast<uint16_t *>(dst + 2 * x) = (uint16_t)(r[g] & 0xffffu);
                            if (x + 1 < X) *reinterpret_cast<uint16_t *>(dst + 2 * x + 2) = (uint16_t)(r[g] >> 16);
                        }
                    }
                }
            }
        }
        __syncthreads();

        // ------------------------------------------------------------ write island records and pool rows
        const Agg excl = ctrl->excl, agg = ctrl->agg;
        if (!excl.poison && !(a.flags & DAQ_SKIP_ISLANDS)) {
            // pool: rows [excl.m, excl.m + agg.m) <- stage, byte range [gs, ge)
            const long long rb = 2ll * X;
            const long long cap_b = a.pool_cap * rb;
            const long long gs = excl.m * rb;
            long long ge = gs + agg.m * rb;
            if (ge > cap_b) {
                ge = cap_b;
                if (tid == 0) atomicOr(reinterpret_cast<unsigned long long *>(&a.counts[2]),
                                       (unsigned long long)DAQ_DEV_POOL_OVERFLOW);
            }
            if (ge > gs) {
                unsigned char *g = reinterpret_cast<unsigned char *>(a.pool);
                long long a16 = (gs + 15) & ~15ll, b16 = ge & ~15ll;
                if (a16 > ge) a16 = ge;
                if (b16 < a16) b16 = a16;
                // head and tail, 2 bytes at a time
                const int n_head = (int)((a16 - gs) >> 1), n_tail = (int)((ge - b16) >> 1);
                if (tid < n_head)
                    *reinterpret_cast<uint16_t *>(g + gs + 2 * tid) =
                        *reinterpret_cast<const uint16_t *>(stage + 2 * tid);
                else if (tid >= 32 && tid < 32 + n_tail) {
                    const long long o = b16 + 2 * (tid - 32);
                    *reinterpret_cast<uint16_t *>(g + o) = *reinterpret_cast<const uint16_t *>(stage + (o - gs));
                }
                // body: 16-byte chunks; stage offset of global a16 is e = a16 - gs (even, < 16)
                const int e = (int)(a16 - gs);
                const long long n_chunks = (b16 - a16) >> 4;
                const int o = e >> 2;
                const bool half = (e & 2) != 0;
                for (long long i = tid; i < n_chunks; i += kThreads) {
                    const uint4 w0 = *reinterpret_cast<const uint4 *>(stage + 16 * i);
                    uint32_t out0, out1, out2, out3;
                    if (e == 0) {
                        out0 = w0.x; out1 = w0.y; out2 = w0.z; out3 = w0.w;
                    } else {
                        const uint4 w1 = *reinterpret_cast<const uint4 *>(stage + 16 * i + 16);
                        uint32_t w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                        uint32_t s0, s1, s2, s3, s4;
                        switch (o) {
                        case 0: s0 = w[0]; s1 = w[1]; s2 = w[2]; s3 = w[3]; s4 = w[4]; break;
                        case 1: s0 = w[1]; s1 = w[2]; s2 = w[3]; s3 = w[4]; s4 = w[5]; break;
                        case 2: s0 = w[2]; s1 = w[3]; s2 = w[4]; s3 = w[5]; s4 = w[6]; break;
                        default: s0 = w[3]; s1 = w[4]; s2 = w[5]; s3 = w[6]; s4 = w[7]; break;
                        }
                        if (half) {
                            out0 = __funnelshift_r(s0, s1, 16);
                            out1 = __funnelshift_r(s1, s2, 16);
                            out2 = __funnelshift_r(s2, s3, 16);
                            out3 = __funnelshift_r(s3, s4, 16);
                        } else {
                            out0 = s0; out1 = s1; out2 = s2; out3 = s3;
                        }
                    }
                    st_global_cs_v4(g + a16 + 16 * i, out0, out1, out2, out3);
                }
            }
            // island records: one per island end in this tile
            if (warp == 0 && lane < NWT) {
                uint32_t E = w_e[lane];
                const uint32_t Mt = w_m[lane], St = w_s[lane];
                bool over = false;
                while (E) {
                    const int b = __ffs(E) - 1;
                    E &= E - 1u;
                    const uint32_t upto = b == 31 ? 0xffffffffu : ((2u << b) - 1u);
                    const uint32_t su = St & upto;
                    const long long idx = excl.s + w_sb[lane] + __popc(su) - 1;
                    const int lrel = su ? 32 * lane + 31 - __clz(su) : w_ls[lane];
                    const long long start = lrel >= 0 ? t0 + lrel : t0 - excl.tr;
                    const long long t_e = t0 + 32 * lane + b;
                    const long long ilen = t_e - start + 1;
                    const long long row_end = excl.m + w_mb[lane] + __popc(Mt & upto) - 1;
                    if (idx < a.hdr_cap) {
                        daq_island *h = a.hdr + idx;
                        h->fill = a.fill_base + f;
                        h->calo = c;
                        h->start = (int32_t)start;
                        h->len = (int32_t)ilen;
                        h->pool_row = row_end - ilen + 1;
                    } else {
                        over = true;
                    }
                }
                if (over) atomicOr(reinterpret_cast<unsigned long long *>(&a.counts[2]),
                                   (unsigned long long)DAQ_DEV_HDR_OVERFLOW);
            }
        }
        if (tid == 0 && tile == a.fill_tile_start[a.n_fills] - 1) {
            const Agg tot = combine(excl, agg);
            a.counts[0] = tot.s;
            a.counts[1] = tot.m;
            a.counts[3] = tile + 1;
            if (tot.m > a.pool_cap && (a.flags & DAQ_SKIP_ISLANDS) == 0)
                atomicOr(reinterpret_cast<unsigned long long *>(&a.counts[2]), (unsigned long long)DAQ_DEV_POOL_OVERFLOW);
            if (tot.s > a.hdr_cap && (a.flags & DAQ_SKIP_ISLANDS) == 0)
                atomicOr(reinterpret_cast<unsigned long long *>(&a.counts[2]), (unsigned long long)DAQ_DEV_HDR_OVERFLOW);
        }
        // the ticket read at the top of the next iteration is behind a __syncthreads
    }
}

// ============================================================================ host side
static size_t tile_smem_bytes(int tw, int X, int rs, int need_sarr)
{
    size_t b = (size_t)X * rs + rs;
    b += (size_t)(((tw * 2 * X + 32) + 15) & ~15);
    b += 128;
    b += (size_t)(tw / 8) * 4;
    b += need_sarr ? (size_t)tw * 4 : 0;
    b += (size_t)(tw / 32) * 4 * 6;
    b += 16 + sizeof(TileCtrl) + 16 + 16;
    return (b + 127) & ~size_t(127);
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

struct Plan {
    int tw, hl, hr, ew, rs, need_sarr;
    size_t smem;
    int64_t max_tiles;
};

static int choose_tile(int requested, int pre, int post)
{
    const int hl = (post + 1 + 7) & ~7, hr = (pre + 1 + 7) & ~7;
    auto fits = [&](int tw) { return tw + hl + hr <= kMaxExtBits; };
    if (requested == 0) {
        for (int tw : {448, 224, 128})
            if (fits(tw)) return tw;
        return -1;
    }
    if (requested != 128 && requested != 224 && requested != 448 && requested != 960) return -1;
    return fits(requested) ? requested : -1;
}

static int make_plan(int n_calo, int n_xtal, int64_t n_samples, int n_fills, const daq_params *p, Plan *pl)
{
    if (!p || n_calo < 0 || n_fills < 0 || n_samples < 0 || n_xtal < 1) return DAQ_EINVAL;
    if (n_xtal > kMaxXtal) return DAQ_EUNSUPPORTED;
    if (p->pre < 0 || p->post < 0 || p->pre + p->post > 512 || p->ped_samples < 1) return DAQ_EINVAL;
    if (p->n_decim < 0 || p->n_decim > 2) return DAQ_EINVAL;
    if (n_samples > (int64_t)INT32_MAX) return DAQ_EUNSUPPORTED;
    pl->need_sarr = 0;
    for (int d = 0; d < p->n_decim; ++d) {
        if (p->decim[d] < 1) return DAQ_EINVAL;
        if (p->decim[d] % 8) pl->need_sarr = 1;
    }
    const int tw = choose_tile(p->tile, p->pre, p->post);
    if (tw < 0) return DAQ_EINVAL;
    pl->tw = tw;
    pl->hl = (p->post + 1 + 7) & ~7;
    pl->hr = (p->pre + 1 + 7) & ~7;
    pl->ew = pl->hl + tw + pl->hr;
    int rs = ((pl->ew * 2) + 15) & ~15;
    if (((rs / 16) & 1) == 0) rs += 16;  // odd multiple of 16 bytes: conflict-free ldmatrix rows
    pl->rs = rs;
    pl->smem = tile_smem_bytes(tw, n_xtal, rs, pl->need_sarr);
    pl->max_tiles = (int64_t)n_fills * n_calo * ((n_samples + tw - 1) / tw);
    return DAQ_OK;
}

template <int TW> static cudaError_t launch_tile(const KArgs &a, const Plan &pl, int grid, cudaStream_t s)
{
    static std::mutex mu;
    static size_t configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> g(mu);
        if (dev >= 0 && dev < 64 && configured[dev] < pl.smem) {
            cudaError_t e = cudaFuncSetAttribute(daq_tile_kernel<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)pl.smem);
            if (e != cudaSuccess) return e;
            configured[dev] = pl.smem;
        }
    }
    if (grid <= 0) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, daq_tile_kernel<TW>, kThreads, pl.smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid = per_sm * device_info(dev).sms;
    }
    daq_tile_kernel<TW><<<grid, kThreads, pl.smem, s>>>(a);
    return cudaGetLastError();
}

static int64_t q_bins(int64_t n, int32_t d) { return d > 0 ? (n + d - 1) / d : 0; }

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
    *bytes = ws_layout(n_fills, n_calo, pl.max_tiles).total;
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
    int64_t q_total = 0;
    for (int d = 0; d < p.n_decim; ++d) q_total += q_bins(n_samples, p.decim[d]) * n_calo;
    if (!skip_q && q_total > 0 && !qhist_inout) return DAQ_EINVAL;
    if (reinterpret_cast<uintptr_t>(out->counts) & 7) return DAQ_EINVAL;
    const WsLayout wl = ws_layout(n_fills, n_calo, pl.max_tiles);
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
        qoff += a.qbins[d] * n_calo;
    }
    a.fill_base = p.fill_base;
    a.fill_len = p.fill_len;
    a.flags = p.flags;
    a.hl = pl.hl;
    a.hr = pl.hr;
    a.ew = pl.ew;
    a.rs = pl.rs;
    a.bulk_ok = (n_samples % 8 == 0) && ((reinterpret_cast<uintptr_t>(samples) & 15) == 0);
    a.need_sarr = pl.need_sarr;
    a.max_tiles = pl.max_tiles;
    a.hdr = skip_isl ? nullptr : out->hdr;
    a.hdr_cap = skip_isl ? 0 : out->hdr_cap;
    a.pool = skip_isl ? nullptr : out->pool;
    a.pool_cap = skip_isl ? 0 : out->pool_row_cap;
    a.ped_out = out->pedestal;
    a.counts = out->counts;
    a.q = qhist_inout;
    unsigned char *ws = static_cast<unsigned char *>(p.workspace);
    a.ticket = reinterpret_cast<unsigned int *>(ws + wl.ticket);
    a.fill_tile_start = reinterpret_cast<long long *>(ws + wl.fts);
    a.lens = reinterpret_cast<int32_t *>(ws + wl.lens);
    a.ptot = reinterpret_cast<int32_t *>(ws + wl.ptot);
    a.status = reinterpret_cast<TileStatus *>(ws + wl.status);

    cudaStream_t s = static_cast<cudaStream_t>(p.stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DAQ_ECUDA;
    const DeviceInfo di = device_info(dev);
    if (di.sms <= 0) return DAQ_ECUDA;
    if ((int)pl.smem > di.smem_optin) return DAQ_EUNSUPPORTED;

    cudaEvent_t const *ev = reinterpret_cast<cudaEvent_t const *>(p.events);
    if (ev && cudaEventRecord(ev[0], s) != cudaSuccess) return DAQ_ECUDA;
    const long long n_cf = (long long)n_fills * n_calo;
    const int prep_grid = (int)std::max<long long>(1, std::min<long long>(std::max<long long>(n_cf, 1), 4ll * di.sms));
    daq_prepare_kernel<<<prep_grid, kThreads, 0, s>>>(a, pl.tw);
    if (cudaGetLastError() != cudaSuccess) return DAQ_ECUDA;
    if (ev && cudaEventRecord(ev[1], s) != cudaSuccess) return DAQ_ECUDA;

    int grid = p.grid;
    if (grid < 0) grid = (int)std::max<int64_t>(1, std::min<int64_t>(pl.max_tiles, INT32_MAX));
    if (grid > 0 && pl.max_tiles > 0 && grid > pl.max_tiles) grid = (int)pl.max_tiles;
    if (pl.max_tiles == 0) grid = 1;
    cudaError_t e;
    switch (pl.tw) {
    case 128: e = launch_tile<128>(a, pl, grid, s); break;
    case 224: e = launch_tile<224>(a, pl, grid, s); break;
    case 448: e = launch_tile<448>(a, pl, grid, s); break;
    default: e = launch_tile<960>(a, pl, grid, s); break;
    }
    if (e != cudaSuccess) return DAQ_ECUDA;
    if (ev && cudaEventRecord(ev[2], s) != cudaSuccess) return DAQ_ECUDA;

    if (p.flags & DAQ_SYNC) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return DAQ_ECUDA;
        int64_t h[4];
        if (cudaMemcpy(h, out->counts, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return DAQ_ECUDA;
        return daq_status_from_counts(h);
    }
    return DAQ_OK;
}

int daq_status_from_counts(const int64_t *c)
{
    if (!c) return DAQ_EINVAL;
    if (c[2] & DAQ_DEV_TIMEOUT) return DAQ_ETIMEOUT;
    if (c[2] & DAQ_DEV_BAD_FILL_LEN) return DAQ_EINVAL;
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
    default: return "unknown status";
    }
}

int daq_version(void) { return 100; }

}  // extern "C"
