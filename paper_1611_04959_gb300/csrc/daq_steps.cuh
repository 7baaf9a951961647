// Per-tile steps of the fused DAQ kernels (Sec. 3, Table 2 of arXiv:1611.04959),
// shared by the simple and the pipelined tile kernels.
//
// A tile is TW consecutive samples [t0, t0 + TW) of one calorimeter-fill.  Its
// crystal rows are held in shared memory with a halo: extended column c is
// sample t0 - HL + c, for c in [0, EW), EW = HL + TW + HR.  The extended tile
// is stored as nbox boxes of [n_xtal][boxw] samples (one 2-D TMA box each, box
// k holding columns [k boxw, (k+1) boxw)), box stride box_stride bytes.  The
// row pitch 2 boxw is an odd multiple of 16 bytes, so the eight rows of every
// ldmatrix are conflict-free.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "daq.h"
#include "daq_device.cuh"

namespace daq {

constexpr uint64_t kWaitLimitNs = 4000000000ull;  // bounded device waits (4 s)
constexpr int kMaxXtal = 64;
constexpr int kMaxExtBits = 1024;  // tile + halos: one warp of 32-bit words

// Scan state of one tile: one 16-byte word, written whole (128-bit release
// store) first with the tile's aggregate, later with its inclusive prefix, and
// read whole (128-bit acquire load).
//   lo = (marked samples << 2) | kind
//   hi = (island starts << 33) | (trailing run << 3) | (continues << 2) | kind
// kind: 0 nothing yet, 1 aggregate, 2 inclusive prefix, 3 poisoned prefix.  The
// kind is kept in both halves; a read whose halves disagree is not used.
struct __align__(16) TileStatus {
    unsigned long long lo, hi;
};
constexpr unsigned kKindAgg = 1, kKindInc = 2, kKindPoison = 3;

struct Agg {
    long long m;   // marked samples (pool rows)
    long long s;   // island starts
    long long tr;  // marked samples in the run that ends at the tile's last sample
    int full;      // every sample marked and the run continues from the previous tile
    int poison;
};

__device__ __forceinline__ Agg agg_identity() { return Agg{0, 0, 0, 1, 0}; }

// Prefix p followed by tile t (associative, not commutative).
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

__device__ __forceinline__ Agg shfl_down_agg(const Agg &a, int d)
{
    Agg r;
    r.m = __shfl_down_sync(kFull, a.m, d);
    r.s = __shfl_down_sync(kFull, a.s, d);
    r.tr = __shfl_down_sync(kFull, a.tr, d);
    r.full = __shfl_down_sync(kFull, a.full, d);
    r.poison = __shfl_down_sync(kFull, a.poison, d);
    return r;
}

struct KArgs {
    CUtensorMap tmap;  // samples as a 2-D tensor [F*C*X rows][n_samples], when use_tma
    const int16_t *samples;
    int32_t n_calo, n_xtal, n_fills;
    int64_t n_samples;  // row pitch
    int32_t threshold, pre, post, ped_samples;
    int32_t n_decim, decim[2];
    int64_t qbins[2], qoff[2];
    int32_t fill_base;
    const int32_t *fill_len;
    uint32_t flags;
    int32_t hl, hr, ew, rs;  // halo left/right, extended width, smem row pitch (bytes) = 2 boxw
    int32_t boxw, nbox, box_stride, slot_bytes;
    int32_t use_tma;
    // stage rows: pitch srow bytes; for even n_xtal, wpr words of data per row
    // and a pitch of srow/4 words = 4 (mod 8), so staging stores are conflict-free
    int32_t srow, wpr;
    unsigned long long wpr_mul;  // floor(2^32 / wpr) + 1, for w / wpr (w < 2^16)
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
    unsigned long long *trace;   // NULL or [max_tiles][16] stage stamps
};

__device__ __forceinline__ void trace_stamp(const KArgs &a, long long tile, int k)
{
    if (a.trace) a.trace[tile * 16 + k] = global_ns();
}

__device__ __forceinline__ void trace_value(const KArgs &a, long long tile, int k, unsigned long long v)
{
    if (a.trace) a.trace[tile * 16 + k] = v;
}

__device__ __forceinline__ unsigned sm_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

struct TileInfo {
    long long tile;  // -1: no more tiles
    long long t0, len, t_end;
    int f, c, ptot, pad;
};

// Bit words of the tile proper and their prefix counts.
struct TileWords {
    uint32_t *m, *s, *e;  // marked, island starts, island ends
    int32_t *mb, *sb;     // marked / starts before the word
    int32_t *ls;          // last island start before the word (tile-relative), -1
};

__device__ __forceinline__ void set_status_bit(const KArgs &a, unsigned long long bit)
{
    atomicOr(reinterpret_cast<unsigned long long *>(&a.counts[2]), bit);
}

__device__ __forceinline__ bool aborted(const KArgs &a)
{
    return (ld_relaxed_u64(reinterpret_cast<const unsigned long long *>(&a.counts[2])) & DAQ_DEV_TIMEOUT) != 0;
}

// Map a ticket to its tile.  Tiles are numbered fill by fill, calorimeter by
// calorimeter, then in time; a fill of length len has ceil(len / TW) tiles
// per calorimeter.
template <int TW>
__device__ bool decode_tile(const KArgs &a, long long tile, TileInfo &T, const long long *fts, const int32_t *lens)
{
    const long long total = fts[a.n_fills];
    T.tile = -1;
    if (tile >= total) return false;
    int lo = 0, hi = a.n_fills - 1;  // last fill whose first tile <= tile
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fts[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    const long long len = lens[lo];
    const long long tpc = (len + TW - 1) / TW;
    const long long rem = tile - fts[lo];
    T.tile = tile;
    T.f = lo;
    T.c = (int)(rem / tpc);
    T.t0 = (rem % tpc) * TW;
    T.len = len;
    T.t_end = T.t0 + TW < len ? T.t0 + TW : len;
    T.ptot = a.ptot[(long long)lo * a.n_calo + T.c];
    T.pad = 0;
    return true;
}

// --------------------------------------------------------------------------- crystal sum + threshold
// Shared-memory address of crystal x's 16 bytes at 8-sample block b of a tile
// slot; crystals past n_xtal read a zero row.
__device__ __forceinline__ uint32_t blk_addr(const KArgs &a, uint32_t slot_s, uint32_t zrow_s, int x, int b)
{
    const int c = 8 * b;
    const int k = (c >= a.boxw) + (c >= 2 * a.boxw) + (c >= 3 * a.boxw) + (c >= 4 * a.boxw);  // nbox <= 5
    const int col = c - k * a.boxw;
    if (x >= a.n_xtal) return zrow_s + 2u * (uint32_t)col;
    return slot_s + (uint32_t)(k * a.box_stride + x * a.rs + 2 * col);
}

// Two 8-sample blocks at once (b1 < 0: only b0), warp-wide: crystal sums,
// threshold bits and block sums.  Lane L of the ldmatrix transposes holds
// crystals 8g + 2(L%4), +1 at sample L/4 of a block; dp2a adds both halves and
// two shuffles finish the crystal sum.  Both blocks' loads are issued first.
__device__ __forceinline__ void sum_block2(const KArgs &a, const TileInfo &T, uint32_t slot_s, uint32_t zrow_s,
                                           bool two_groups, int b0, int b1, int nbt, uint8_t *abyte,
                                           int32_t *blocksum, int32_t *sarr, int lane)
{
    uint32_t r[2][8];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int k = 0; k < 8; ++k) r[u][k] = 0u;
    ldsm_x4_trans(blk_addr(a, slot_s, zrow_s, lane, b0), r[0][0], r[0][1], r[0][2], r[0][3]);
    if (two_groups) ldsm_x4_trans(blk_addr(a, slot_s, zrow_s, lane + 32, b0), r[0][4], r[0][5], r[0][6], r[0][7]);
    if (b1 >= 0) {
        ldsm_x4_trans(blk_addr(a, slot_s, zrow_s, lane, b1), r[1][0], r[1][1], r[1][2], r[1][3]);
        if (two_groups)
            ldsm_x4_trans(blk_addr(a, slot_s, zrow_s, lane + 32, b1), r[1][4], r[1][5], r[1][6], r[1][7]);
    }
    const int j = lane >> 2;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int b = u == 0 ? b0 : b1;
        if (b < 0) break;
        int acc = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc = __dp2a_lo((int)r[u][k], 0x0101, acc);
        acc += __shfl_xor_sync(kFull, acc, 1);
        acc += __shfl_xor_sync(kFull, acc, 2);
        const long long t = T.t0 - a.hl + 8 * b + j;
        const int S = acc - T.ptot;
        const bool cross = (t >= 0) && (t < T.len) && (S > a.threshold);
        uint32_t v = __ballot_sync(kFull, cross) & 0x11111111u;
        v = (v | (v >> 3)) & 0x03030303u;
        v = (v | (v >> 6)) & 0x000f000fu;
        v = (v | (v >> 12)) & 0xffu;
        if (lane == 0) abyte[b] = (uint8_t)v;
        const int bt = b - a.hl / 8;
        if (bt >= 0 && bt < nbt) {
            const bool in = t < T.t_end;
            int sv = in ? S : 0;
            sv += __shfl_xor_sync(kFull, sv, 4);
            sv += __shfl_xor_sync(kFull, sv, 8);
            sv += __shfl_xor_sync(kFull, sv, 16);
            if (lane == 0) blocksum[bt] = sv;
            if (a.need_sarr && (lane & 3) == 0 && in) sarr[8 * bt + j] = S;
        }
    }
}

// Marks of the 32 extended-tile bits held by this lane: M[i] = OR of A over
// [i - post, i + pre].  Fast form (post + pre <= 96): the lane gathers the seven
// threshold words around its own once and widens them in registers.
__device__ __forceinline__ uint32_t marks_word(const KArgs &a, uint32_t A, int lane)
{
    const int L = a.pre + a.post + 1;
    if (a.pre + a.post <= 96) {
        uint32_t win[8];
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const int src = lane + i - 3;
            const uint32_t v = __shfl_sync(kFull, A, src & 31);
            win[i] = (src >= 0 && src < 32) ? v : 0u;
        }
        win[7] = 0u;
        // V = bits [32 lane - post, 32 lane - post + 128) of the threshold array
        const int o = 96 - a.post, qw = o >> 5, sw = o & 31;
        // drop the qw lowest words (uniform qw in 0..3) with constant-index moves
        if (qw & 2) {
#pragma unroll
            for (int k = 0; k < 6; ++k) win[k] = win[k + 2];
            win[6] = win[7] = 0u;
        }
        if (qw & 1) {
#pragma unroll
            for (int k = 0; k < 7; ++k) win[k] = win[k + 1];
            win[7] = 0u;
        }
        uint32_t v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = sw ? __funnelshift_r(win[i], win[i + 1], sw) : win[i];
        unsigned long long rlo = ((unsigned long long)v[1] << 32) | v[0];
        unsigned long long rhi = ((unsigned long long)v[3] << 32) | v[2];
        auto shr128 = [](unsigned long long &lo, unsigned long long &hi, int sft) {
            if (sft >= 64) {
                lo = hi >> (sft - 64);
                hi = 0ull;
            } else if (sft > 0) {
                lo = (lo >> sft) | (hi << (64 - sft));
                hi >>= sft;
            }
        };
        // OR of L consecutive bits by doubling
        int cov = 1;
        while (2 * cov <= L) {
            unsigned long long tlo = rlo, thi = rhi;
            shr128(tlo, thi, cov);
            rlo |= tlo;
            rhi |= thi;
            cov *= 2;
        }
        if (cov < L) {
            unsigned long long tlo = rlo, thi = rhi;
            shr128(tlo, thi, L - cov);
            rlo |= tlo;
        }
        return (uint32_t)rlo;
    }
    // general form: forward spread by post, backward spread by pre, across the warp
    uint32_t Fv = A;
    int cov = 1;
    while (2 * cov <= a.post + 1) {
        Fv |= shl_bits(Fv, cov, lane);
        cov *= 2;
    }
    if (cov < a.post + 1) Fv |= shl_bits(Fv, a.post + 1 - cov, lane);
    uint32_t Mv = Fv;
    cov = 1;
    while (2 * cov <= a.pre + 1) {
        Mv |= shr_bits(Mv, cov, lane);
        cov *= 2;
    }
    if (cov < a.pre + 1) Mv |= shr_bits(Mv, a.pre + 1 - cov, lane);
    return Mv;
}

// --------------------------------------------------------------------------- windows + merge (one warp)
// From the threshold bits of the extended tile: marks M (crossings widened by
// pre/post samples), island starts and ends inside the tile, prefix counts per
// word, and the tile's aggregate for the cross-tile scan.
template <int TW>
__device__ __forceinline__ Agg tile_bits(const KArgs &a, const TileInfo &T, const uint8_t *abyte, TileWords w,
                                         int lane)
{
    constexpr int NWT = TW / 32;
    const int HL = a.hl;
    const int NWE = (a.ew + 31) / 32;
    const long long e0 = T.t0 - HL;
    const uint32_t A = lane < NWE ? reinterpret_cast<const uint32_t *>(abyte)[lane] : 0u;
    uint32_t Mv = marks_word(a, A, lane);
    Mv &= range_mask(32ll * lane, -e0, T.len - e0);  // only samples of [0, len) are marked
    const uint32_t prev_w = __shfl_sync(kFull, Mv, (HL - 1) >> 5);
    const uint32_t next_w = __shfl_sync(kFull, Mv, (HL + TW) >> 5);
    const int qo = HL >> 5, sh = HL & 31;
    uint32_t lo_w = __shfl_down_sync(kFull, Mv, qo);
    uint32_t hi_w = __shfl_down_sync(kFull, Mv, qo + 1 < 32 ? qo + 1 : 31);
    const uint32_t m_prev = (prev_w >> ((HL - 1) & 31)) & 1u;
    const uint32_t m_next = (next_w >> ((HL + TW) & 31)) & 1u;
    if (lane + qo > 31) lo_w = 0u;
    if (lane + qo + 1 > 31) hi_w = 0u;
    uint32_t Mt = sh ? ((lo_w >> sh) | (hi_w << (32 - sh))) : lo_w;
    if (lane >= NWT) Mt = 0u;
    uint32_t below = __shfl_up_sync(kFull, Mt, 1);
    uint32_t above = __shfl_down_sync(kFull, Mt, 1);
    if (lane == 0) below = m_prev << 31;
    if (lane == NWT - 1) above = m_next;
    if (lane >= NWT) above = 0u;
    const uint32_t St = Mt & ~((Mt << 1) | (below >> 31));
    const uint32_t Et = Mt & ~((Mt >> 1) | (above << 31));
    // one scan for both counts (each <= 1024): marked in the low half, starts in the high half
    const uint32_t packed = (uint32_t)__popc(Mt) | ((uint32_t)__popc(St) << 16);
    uint32_t x = packed;
    int mx = St ? 32 * lane + 31 - __clz(St) : -1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        const int ym = __shfl_up_sync(kFull, mx, d);
        if (lane >= d) {
            x += y;
            mx = max(mx, ym);
        }
    }
    const uint32_t tot = __shfl_sync(kFull, x, 31);
    const int ls_incl_prev = __shfl_up_sync(kFull, mx, 1);
    const uint32_t excl = x - packed;
    const int ls = lane == 0 ? -1 : ls_incl_prev;
    const int nt = (int)(T.t_end - T.t0);
    const uint32_t zeros = ~Mt & range_mask(32ll * lane, 0, nt);
    const int lz = (int)__reduce_max_sync(kFull, zeros ? (unsigned)(32 * lane + 32 - __clz(zeros)) : 0u) - 1;
    if (lane < NWT) {
        w.m[lane] = Mt;
        w.s[lane] = St;
        w.e[lane] = Et;
        w.mb[lane] = (int)(excl & 0xffffu);
        w.sb[lane] = (int)(excl >> 16);
        w.ls[lane] = ls;
    }
    Agg agg;
    agg.m = tot & 0xffffu;
    agg.s = tot >> 16;
    agg.tr = nt - 1 - lz;
    agg.full = (lz < 0) && m_prev;
    agg.poison = 0;
    return agg;
}

// --------------------------------------------------------------------------- cross-tile scan
__device__ __forceinline__ void publish(TileStatus *st, long long tile, bool inclusive, const Agg &v)
{
    const unsigned long long kind = inclusive ? (v.poison ? kKindPoison : kKindInc) : kKindAgg;
    const unsigned long long lo = ((unsigned long long)v.m << 2) | kind;
    const unsigned long long hi = ((unsigned long long)v.s << 33) | ((unsigned long long)v.tr << 3) |
                                  ((unsigned long long)(v.full != 0) << 2) | kind;
    st_release_b128(&st[tile], lo, hi);
}

// kind of a status read (0 when not yet published or the halves disagree)
__device__ __forceinline__ unsigned read_status(const TileStatus *st, long long idx, Agg &v)
{
    unsigned long long lo, hi;
    // relaxed: the 16-byte word is the whole message, nothing else is read on its account
    ld_relaxed_b128(&st[idx], lo, hi);
    const unsigned k = (unsigned)(lo & 3ull);
    if (k == 0 || k != (unsigned)(hi & 3ull)) return 0;
    v.m = (long long)(lo >> 2);
    v.s = (long long)(hi >> 33);
    v.tr = (long long)((hi >> 3) & 0x3fffffffull);
    v.full = (int)((hi >> 2) & 1ull);
    v.poison = k == kKindPoison;
    return k;
}

// Decoupled look-back (one warp): exclusive prefix of `tile` over all earlier
// tiles.  Each round reads 128 predecessors (4 per lane, one 16-byte load
// each).  It stops at the nearest inclusive prefix (g = stop, counting back
// from the latest); the window's combination is formed with warp reductions:
// marked and start counts add up, and the trailing run adds the runs of the
// latest entries up to and including the first one that is not fully marked.
// Bounded: gives up after kWaitLimitNs or once another CTA has flagged a
// timeout, returning a poisoned prefix.
__device__ Agg look_back(const KArgs &a, long long tile, int lane, unsigned *stats = nullptr)
{
    constexpr int PER = 4, BIG = 1 << 20;
    const TileStatus *st = a.status;
    long long pos = tile - 1;
    Agg acc = agg_identity();
    uint64_t t_start = 0;
    bool waiting = false;
    unsigned rounds = 0, waits = 0;
    for (uint32_t iter = 0;; ++iter) {
        unsigned kind[PER];
        Agg v[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const long long idx = pos - (PER * lane + j);
            v[j] = agg_identity();
            v[j].full = 0;
            kind[j] = kKindInc;  // before tile 0: an empty inclusive prefix
            if (idx >= 0) kind[j] = read_status(st, idx, v[j]);
        }
        int my_stop = BIG, my_miss = BIG;
#pragma unroll
        for (int j = PER - 1; j >= 0; --j) {
            if (kind[j] >= kKindInc) my_stop = PER * lane + j;
            if (kind[j] == 0) my_miss = PER * lane + j;
        }
        const int stop = (int)__reduce_min_sync(kFull, (unsigned)my_stop);
        const int missing = (int)__reduce_min_sync(kFull, (unsigned)my_miss);
        const int last = stop < BIG ? stop : 32 * PER - 1;
        if (missing <= last) {
            // a needed predecessor has published nothing yet: wait (bounded)
            ++waits;
            if (!waiting) {
                t_start = global_ns();
                waiting = true;
            }
            if ((iter & 15u) == 15u) {
                int give_up = lane == 0 && (global_ns() - t_start > kWaitLimitNs || aborted(a));
                if (__shfl_sync(kFull, give_up, 0)) {
                    acc.poison = 1;
                    if (lane == 0) set_status_bit(a, DAQ_DEV_TIMEOUT);
                    return acc;
                }
            }
            __nanosleep(100);
            continue;
        }
        // first entry (from the latest) that is not fully marked, within [0, last]
        int my_nf = BIG;
#pragma unroll
        for (int j = PER - 1; j >= 0; --j)
            if (PER * lane + j <= last && !v[j].full) my_nf = PER * lane + j;
        const int nf = (int)__reduce_min_sync(kFull, (unsigned)my_nf);
        const int gstar = nf < last ? nf : last;
        unsigned m_agg = 0, s_agg = 0, tr_sum = 0;
        long long m_inc = 0, s_inc = 0;
        int poison = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int g = PER * lane + j;
            if (g > last) continue;
            if (g == stop) {
                m_inc = v[j].m;
                s_inc = v[j].s;
            } else {
                m_agg += (unsigned)v[j].m;  // aggregates: at most 127 tiles of <= 960 samples
                s_agg += (unsigned)v[j].s;
            }
            if (g <= gstar) tr_sum += (unsigned)v[j].tr;
            poison |= v[j].poison;
        }
        Agg window;
        window.m = (long long)__reduce_add_sync(kFull, m_agg);
        window.s = (long long)__reduce_add_sync(kFull, s_agg);
        window.tr = (long long)__reduce_add_sync(kFull, tr_sum);
        window.full = nf > last;
        window.poison = __any_sync(kFull, poison);
        if (stop < BIG) {
            const int src = stop / PER;
            window.m += __shfl_sync(kFull, m_inc, src);
            window.s += __shfl_sync(kFull, s_inc, src);
        }
        acc = combine(window, acc);
        ++rounds;
        if (stop < BIG) {
            if (stats) *stats = rounds * 100000u + waits;
            return acc;
        }
        pos -= 32 * PER;
        waiting = false;
    }
}

// --------------------------------------------------------------------------- staging of pool rows
// Block bt of the tile proper (warp-wide): every marked sample's n_xtal raw
// values go to its row in the tile-local stage area (row = marked samples
// before it in the tile).
__device__ __forceinline__ void stage_block(const KArgs &a, uint32_t slot_s, uint32_t zrow_s, bool two_groups,
                                            int bt, const uint32_t *w_m, const int32_t *w_mb, unsigned char *stage,
                                            int lane)
{
    const int X = a.n_xtal;
    const int w = bt >> 2, shift = (bt & 3) * 8;
    const uint32_t mw = w_m[w];
    const uint32_t bits = (mw >> shift) & 0xffu;
    if (!bits) return;
    const int b = bt + a.hl / 8;
    uint32_t r[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    ldsm_x4_trans(blk_addr(a, slot_s, zrow_s, lane, b), r[0], r[1], r[2], r[3]);
    if (two_groups) ldsm_x4_trans(blk_addr(a, slot_s, zrow_s, lane + 32, b), r[4], r[5], r[6], r[7]);
    const int j = lane >> 2, q4 = lane & 3;
    if (!((bits >> j) & 1u)) return;
    const int rl = w_mb[w] + __popc(mw & ((1u << (shift + j)) - 1u));
    unsigned char *dst = stage + (size_t)rl * a.srow;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const int x = 8 * g + 2 * q4;
        if ((g >= 4 && !two_groups) || x >= X) continue;
        if (x + 1 < X && !(X & 1)) {
            *reinterpret_cast<uint32_t *>(dst + 2 * x) = r[g];
        } else {
            *reinterpret_cast<uint16_t *>(dst + 2 * x) = (uint16_t)(r[g] & 0xffffu);
            if (x + 1 < X) *reinterpret_cast<uint16_t *>(dst + 2 * x + 2) = (uint16_t)(r[g] >> 16);
        }
    }
}

// --------------------------------------------------------------------------- pool rows to global
// 16 bytes starting e bytes (even, < 16) into the 32 bytes at p (16-aligned).
__device__ __forceinline__ uint4 shifted_chunk(const unsigned char *p, int e)
{
    const uint4 w0 = *reinterpret_cast<const uint4 *>(p);
    if (e == 0) return w0;
    const uint4 w1 = *reinterpret_cast<const uint4 *>(p + 16);
    uint32_t s0, s1, s2, s3, s4;
    switch (e >> 2) {
    case 0: s0 = w0.x; s1 = w0.y; s2 = w0.z; s3 = w0.w; s4 = w1.x; break;
    case 1: s0 = w0.y; s1 = w0.z; s2 = w0.w; s3 = w1.x; s4 = w1.y; break;
    case 2: s0 = w0.z; s1 = w0.w; s2 = w1.x; s3 = w1.y; s4 = w1.z; break;
    default: s0 = w0.w; s1 = w1.x; s2 = w1.y; s3 = w1.z; s4 = w1.w; break;
    }
    if (e & 2)
        return make_uint4(__funnelshift_r(s0, s1, 16), __funnelshift_r(s1, s2, 16), __funnelshift_r(s2, s3, 16),
                          __funnelshift_r(s3, s4, 16));
    return make_uint4(s0, s1, s2, s3);
}

// Rows [excl.m, excl.m + agg.m) from the stage area (a group of nthr threads,
// id gt).  The body goes out in aligned 16-byte stores; the head and tail
// (< 16 bytes each, shared with neighbouring tiles' rows) in 2-byte stores.
// Even n_xtal: rows are wpr words; stage row r holds them at word r * P (P =
// srow / 4), so output word w comes from stage word (w / wpr) * P + w % wpr.
__device__ __forceinline__ void copy_out_words(const KArgs &a, const unsigned char *stage, const Agg &excl,
                                               const Agg &agg, int gt, int nthr)
{
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(stage);
    const int P = a.srow >> 2, wpr = a.wpr;
    const long long G0 = excl.m * wpr;  // global word of the tile's first output word
    long long n_words = agg.m * wpr;
    const long long cap_w = a.pool_cap * wpr;
    if (G0 + n_words > cap_w) {
        n_words = cap_w - G0;
        if (gt == 0) set_status_bit(a, DAQ_DEV_POOL_OVERFLOW);
    }
    if (n_words <= 0) return;
    uint32_t *g32 = reinterpret_cast<uint32_t *>(a.pool) + G0;
    auto row_of = [&](uint32_t w) {
        uint32_t r = (uint32_t)(((unsigned long long)w * a.wpr_mul) >> 32);
        if (r * (uint32_t)wpr > w) --r;
        return r;
    };
    auto src = [&](uint32_t w) {
        const uint32_t r = row_of(w);
        return r * (uint32_t)P + (w - r * (uint32_t)wpr);
    };
    const int head = (int)min((long long)((4 - (G0 & 3)) & 3), n_words);
    const long long n_chunks = (n_words - head) >> 2;
    const long long tail0 = head + 4 * n_chunks;
    const int n_tail = (int)(n_words - tail0);
    if (gt < head) g32[gt] = sw[src((uint32_t)gt)];
    else if (gt >= 4 && gt < 4 + n_tail) g32[tail0 + gt - 4] = sw[src((uint32_t)(tail0 + gt - 4))];
    constexpr int U = 4;
    for (long long c0 = gt; c0 < n_chunks; c0 += (long long)U * nthr) {
        uint4 out[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long c = c0 + (long long)u * nthr;
            out[u] = make_uint4(0u, 0u, 0u, 0u);
            if (c < n_chunks) {
                const uint32_t w = (uint32_t)(head + 4 * c);
                const uint32_t r = row_of(w);
                uint32_t k = w - r * (uint32_t)wpr, base = r * (uint32_t)P;
                uint32_t vals[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    vals[e] = sw[base + k];
                    if (++k == (uint32_t)wpr) {
                        k = 0;
                        base += P;
                    }
                }
                out[u] = make_uint4(vals[0], vals[1], vals[2], vals[3]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long c = c0 + (long long)u * nthr;
            if (c < n_chunks) st_global_cs_v4(g32 + head + 4 * c, out[u].x, out[u].y, out[u].z, out[u].w);
        }
    }
}

__device__ __forceinline__ void copy_out(const KArgs &a, const unsigned char *stage, const Agg &excl,
                                         const Agg &agg, int gt, int nthr)
{
    if (!(a.n_xtal & 1)) {
        copy_out_words(a, stage, excl, agg, gt, nthr);
        return;
    }
    const long long rb = 2ll * a.n_xtal;
    const long long cap_b = a.pool_cap * rb;
    const long long gs = excl.m * rb;
    long long ge = gs + agg.m * rb;
    if (ge > cap_b) {
        ge = cap_b;
        if (gt == 0) set_status_bit(a, DAQ_DEV_POOL_OVERFLOW);
    }
    if (ge <= gs) return;
    unsigned char *g = reinterpret_cast<unsigned char *>(a.pool);
    long long a16 = (gs + 15) & ~15ll, b16 = ge & ~15ll;
    if (a16 > ge) a16 = ge;
    if (b16 < a16) b16 = a16;
    const int n_head = (int)((a16 - gs) >> 1), n_tail = (int)((ge - b16) >> 1);
    if (gt < n_head)
        *reinterpret_cast<uint16_t *>(g + gs + 2 * gt) = *reinterpret_cast<const uint16_t *>(stage + 2 * gt);
    else if (gt >= 8 && gt < 8 + n_tail) {
        const long long o = b16 + 2 * (gt - 8);
        *reinterpret_cast<uint16_t *>(g + o) = *reinterpret_cast<const uint16_t *>(stage + (o - gs));
    }
    const int e = (int)(a16 - gs);  // stage offset of global a16: even, < 16
    const long long n_chunks = (b16 - a16) >> 4;
    constexpr int U = 4;  // chunks per thread per round: loads first, then stores
    for (long long i0 = gt; i0 < n_chunks; i0 += (long long)U * nthr) {
        uint4 out[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = i0 + (long long)u * nthr;
            if (i < n_chunks) out[u] = shifted_chunk(stage + 16 * i, e);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = i0 + (long long)u * nthr;
            if (i < n_chunks) st_global_cs_v4(g + a16 + 16 * i, out[u].x, out[u].y, out[u].z, out[u].w);
        }
    }
}

// --------------------------------------------------------------------------- island records (one warp)
// One record per island end inside the tile.  An island that began in an
// earlier tile starts at t0 - excl.tr (the marked run entering the tile).
template <int TW>
__device__ __forceinline__ void write_headers(const KArgs &a, const TileInfo &T, TileWords w, const Agg &excl,
                                              int lane)
{
    constexpr int NWT = TW / 32;
    if (lane >= NWT) return;
    uint32_t E = w.e[lane];
    const uint32_t Mt = w.m[lane], St = w.s[lane];
    bool over = false;
    while (E) {
        const int b = __ffs(E) - 1;
        E &= E - 1u;
        const uint32_t upto = b == 31 ? 0xffffffffu : ((2u << b) - 1u);
        const uint32_t su = St & upto;
        const long long idx = excl.s + w.sb[lane] + __popc(su) - 1;
        const int lrel = su ? 32 * lane + 31 - __clz(su) : w.ls[lane];
        const long long start = lrel >= 0 ? T.t0 + lrel : T.t0 - excl.tr;
        const long long t_e = T.t0 + 32 * lane + b;
        const long long ilen = t_e - start + 1;
        const long long row_end = excl.m + w.mb[lane] + __popc(Mt & upto) - 1;
        if (idx < a.hdr_cap) {
            daq_island *h = a.hdr + idx;
            h->fill = a.fill_base + T.f;
            h->calo = T.c;
            h->start = (int32_t)start;
            h->len = (int32_t)ilen;
            h->pool_row = row_end - ilen + 1;
        } else {
            over = true;
        }
    }
    if (over) set_status_bit(a, DAQ_DEV_HDR_OVERFLOW);
}

// --------------------------------------------------------------------------- Q decimation + fill sum
// Partial bins of the tile (a group of nthr threads): B_D[k] restricted to the
// tile, added atomically to the calorimeter's int64 histogram.
__device__ __forceinline__ void q_partial(const KArgs &a, const TileInfo &T, const int32_t *blocksum,
                                          const int32_t *sarr, int gt, int nthr)
{
    for (int d = 0; d < a.n_decim; ++d) {
        const long long D = a.decim[d];
        unsigned long long *qrow =
            reinterpret_cast<unsigned long long *>(a.q + a.qoff[d] + (long long)T.c * a.qbins[d]);
        const long long k_lo = T.t0 / D, k_hi = (T.t_end - 1) / D;
        for (long long k = k_lo + gt; k <= k_hi; k += nthr) {
            const long long lo = (k * D > T.t0 ? k * D : T.t0) - T.t0;
            const long long hi = (k * D + D < T.t_end ? k * D + D : T.t_end) - T.t0;
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

// Counts of the whole call, from the last tile's inclusive prefix.
__device__ __forceinline__ void write_counts(const KArgs &a, long long tile, const Agg &incl)
{
    a.counts[0] = incl.s;
    a.counts[1] = incl.m;
    a.counts[3] = tile + 1;
    if (!(a.flags & DAQ_SKIP_ISLANDS)) {
        if (incl.m > a.pool_cap) set_status_bit(a, DAQ_DEV_POOL_OVERFLOW);
        if (incl.s > a.hdr_cap) set_status_bit(a, DAQ_DEV_HDR_OVERFLOW);
    }
}

}  // namespace daq
