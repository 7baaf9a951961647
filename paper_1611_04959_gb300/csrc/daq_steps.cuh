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
constexpr int kMaxTileWords = 14;                 // marks words of the widest two-pass tile (448 samples)
// kernels a call may use (daq_params.grid picks one)
enum : int32_t { kModeTwoPass = 0, kModePlain = 1, kModePipelined = 2, kModeFused = 3, kModeStream = 4, kModePark = 5 };
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

__device__ __forceinline__ Agg shfl_up_agg(const Agg &a, int d)
{
    Agg r;
    r.m = __shfl_up_sync(kFull, a.m, d);
    r.s = __shfl_up_sync(kFull, a.s, d);
    r.tr = __shfl_up_sync(kFull, a.tr, d);
    r.full = __shfl_up_sync(kFull, a.full, d);
    r.poison = __shfl_up_sync(kFull, a.poison, d);
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
    CUtensorMap tmap;    // samples as a 2-D tensor [F*C*X rows][n_samples], when use_tma: boxes with halo
    CUtensorMap tmap_b;  // the same tensor, boxes of the compact pass (tile proper only)
    CUtensorMap tmap_c;  // the same tensor, 64-sample boxes (the streaming form's compaction steps)
    const int16_t *samples;
    int32_t n_calo, n_xtal, n_fills;
    int64_t n_samples;  // row pitch
    int32_t threshold, pre, post, ped_samples;
    int32_t n_decim, decim[2];
    int64_t qbins[2], qoff[2];
    int32_t fill_base, calo_base;
    int32_t q_calos;  // calorimeter rows of each decimation's block of Q
    uint64_t wait_ns;  // limit of waits on other CTAs' published state
    const int32_t *fill_len;
    uint32_t flags;
    int32_t hl, hr, ew, rs;  // halo left/right, extended width, smem row pitch (bytes) = 2 boxw
    int32_t boxw, nbox, box_stride, slot_bytes;
    int32_t boxw_b, nbox_b, box_stride_b, slot_bytes_b, rs_b;  // compact pass: tile proper only
    int32_t use_tma;
    int32_t mode;
    // two-pass form: the count pass loads the tile proper only (hl = hr = 0)
    // and stores internal marks and crossings; the scan completes the marks
    int32_t halo_free;
    // stage rows: pitch srow bytes = P words, P the first odd number >= ceil(n_xtal/2)
    // (odd, so that the two rows a warp's staging store writes fall in 2-way
    // conflicts at worst); for even n_xtal, wpr = n_xtal/2 words of data per row
    int32_t srow, wpr;
    unsigned long long wpr_mul;  // floor(2^32 / wpr) + 1, for w / wpr (w < 2^16)
    int32_t need_sarr;
    int64_t max_tiles;
    // single-launch form: tiles the count role may run ahead of the compact
    // role, and the two progress counters (tiles scanned, tiles compacted)
    int64_t lag_tiles;
    int32_t str_meta, str_stages;  // streaming and single-read forms: tile records and row stages per CTA
    int32_t pk_slots, pk_cols;     // single-read form: Tensor Memory park slots per CTA, columns per slot
    unsigned long long *fctr;
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
    uint32_t *marks;             // two-pass: [max_tiles][TW/32] marks words of each tile
    void *recs;                  // two-pass: [max_tiles] tile aggregates
    void *excl;                  // two-pass: [max_tiles] exclusive prefixes
    TileStatus *scan_status;     // two-pass: [scan blocks] published aggregate / inclusive prefix of each block
    unsigned int *scan_ticket;   // two-pass: scan block order
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
// want_ptot = false leaves T.ptot at 0 (no global load; for callers that
// issue a bulk copy right after decoding and take the pedestal sum elsewhere).
template <int TW>
__device__ bool decode_tile(const KArgs &a, long long tile, TileInfo &T, const long long *fts, const int32_t *lens,
                            bool want_ptot = true)
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
    T.ptot = want_ptot ? a.ptot[(long long)lo * a.n_calo + T.c] : 0;
    T.pad = 0;
    return true;
}

// --------------------------------------------------------------------------- tile loads
// Issue the TMA box loads of one tile (one thread; the caller armed `bar`).
__device__ __forceinline__ void issue_tile_load(const KArgs &a, const TileInfo &T, unsigned char *slot,
                                                uint64_t *bar)
{
    const int c0 = (int)(T.t0 - a.hl);
    const int c1 = (int)(((long long)T.f * a.n_calo + T.c) * a.n_xtal);
    if (a.mode == kModeFused || a.mode == kModeStream) {  // re-read soon by the compaction: keep them in L2
        const uint64_t pol = l2_policy_evict_last();
        for (int k = 0; k < a.nbox; ++k)
            tma_load_2d_hint(slot + (size_t)k * a.box_stride, &a.tmap, c0 + k * a.boxw, c1, bar, pol);
        return;
    }
    for (int k = 0; k < a.nbox; ++k) tma_load_2d(slot + (size_t)k * a.box_stride, &a.tmap, c0 + k * a.boxw, c1, bar);
}

__device__ __forceinline__ uint32_t tile_load_bytes(const KArgs &a)
{
    return (uint32_t)a.nbox * (uint32_t)a.n_xtal * (uint32_t)a.rs;
}

// Fallback load with plain loads (rows not 16-byte aligned), same layout as the boxes.
__device__ __forceinline__ void plain_tile_load(const KArgs &a, const TileInfo &T, unsigned char *slot, int tid,
                                                int nthr)
{
    const int X = a.n_xtal, W = a.nbox * a.boxw;
    const long long e0 = T.t0 - a.hl;
    const long long cf = (long long)T.f * a.n_calo + T.c;
    const int16_t *rows = a.samples + cf * X * a.n_samples;
    for (int i = tid; i < X * W; i += nthr) {
        const int x = i / W, c = i - x * W;
        const int k = c / a.boxw, col = c - k * a.boxw;
        const long long t = e0 + c;
        int16_t v = 0;
        if (t >= 0 && t < a.n_samples) v = rows[(long long)x * a.n_samples + t];
        *reinterpret_cast<int16_t *>(slot + (size_t)k * a.box_stride + (size_t)x * a.rs + 2 * col) = v;
    }
}

// --------------------------------------------------------------------------- crystal sum + threshold
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Spread the 32 bits of x to the even bit positions of a 64-bit word.
__device__ __forceinline__ unsigned long long spread_bits(uint32_t x)
{
    unsigned long long v = x;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

// One warp step of the sum pass over 64 extended columns [64 it, 64 it + 64):
// lane L owns the two samples of columns c = 64 it + 2L, c + 1, reads their
// word from every crystal row (conflict-free 4-byte loads) and
//   - adds the crystals (dp2a takes each 16-bit half with its sign),
//   - subtracts the summed pedestals and tests the threshold (two ballots give
//     the 64 threshold bits of the step),
//   - adds block sums of 8 samples for the Q histograms,
//   - writes the samples' rows, crystals in order, to the stage area (row =
//     sample - t0, pitch srow), for samples of the tile proper; two byte
//     permutes turn (crystal x, x+1) x (sample t, t+1) into row words.
__device__ __forceinline__ void sum_pass_step(const KArgs &a, const TileInfo &T, uint32_t slot_s, int it,
                                              int nbt, uint8_t *abyte, int32_t *blocksum, int32_t *sarr,
                                              unsigned char *stage, int lane)
{
    const int X = a.n_xtal;
    const int c = 64 * it + 2 * lane;
    const bool have = c < a.ew;  // ew is even, so c + 1 < ew too
    const int k = (c >= a.boxw) + (c >= 2 * a.boxw) + (c >= 3 * a.boxw) + (c >= 4 * a.boxw);
    const uint32_t base = slot_s + (uint32_t)(k * a.box_stride + 2 * (c - k * a.boxw));
    const long long t = T.t0 - a.hl + c;
    const bool st0 = stage && have && t >= T.t0 && t < T.t_end;
    const bool st1 = stage && have && t + 1 >= T.t0 && t + 1 < T.t_end;
    uint32_t *row0 = reinterpret_cast<uint32_t *>(stage + (st0 || st1 ? (t - T.t0) * a.srow : 0));
    uint32_t *row1 = row0 + (a.srow >> 2);
    int acc0 = 0, acc1 = 0;
    if (have) {
        // even and odd crystals in separate accumulators: two dependency chains
        // of X/2 dp2a each instead of one of X
        int acc0b = 0, acc1b = 0;
#pragma unroll 9
        for (int x = 0; x < X; x += 2) {
            const uint32_t w0 = lds_u32(base + (uint32_t)(x * a.rs));
            const uint32_t w1 = x + 1 < X ? lds_u32(base + (uint32_t)((x + 1) * a.rs)) : 0u;
            acc0 = __dp2a_lo((int)w0, 0x0001, acc0);
            acc1 = __dp2a_lo((int)w0, 0x0100, acc1);
            acc0b = __dp2a_lo((int)w1, 0x0001, acc0b);
            acc1b = __dp2a_lo((int)w1, 0x0100, acc1b);
            if (st0) row0[x >> 1] = __byte_perm(w0, w1, 0x5410);
            if (st1) row1[x >> 1] = __byte_perm(w0, w1, 0x7632);
        }
        acc0 += acc0b;
        acc1 += acc1b;
    }
    const int S0 = acc0 - T.ptot, S1 = acc1 - T.ptot;
    const bool in0 = have && t >= 0 && t < T.len, in1 = have && t + 1 >= 0 && t + 1 < T.len;
    const uint32_t be = __ballot_sync(kFull, in0 && S0 > a.threshold);
    const uint32_t bo = __ballot_sync(kFull, in1 && S1 > a.threshold);
    if (lane == 0) {
        const unsigned long long m = spread_bits(be) | (spread_bits(bo) << 1);
        *reinterpret_cast<uint2 *>(abyte + 8 * it) = make_uint2((uint32_t)m, (uint32_t)(m >> 32));
    }
    // block sums of the tile proper: blocks of 8 samples = 4 lanes
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

// Island structure of the tile proper from its marks (one warp; lane w holds
// marks word w, bits [32w, 32w + 32) of the tile, 0 past the tile), the marks
// of the samples just before (m_prev) and after (m_next) the tile, and nt =
// samples in the tile.  Writes starts, ends, per-word prefix counts and the
// last island start before each word (TileWords, nullable), optionally the row
// table (row -> marked sample), and returns the tile's aggregate.
template <int TW>
__device__ __forceinline__ Agg words_from_marks(uint32_t Mt, uint32_t m_prev, uint32_t m_next, int nt,
                                                TileWords w, int16_t *rowtab, int lane)
{
    constexpr int NWT = TW / 32;
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
    const uint32_t zeros = ~Mt & range_mask(32ll * lane, 0, nt);
    const int lz = (int)__reduce_max_sync(kFull, zeros ? (unsigned)(32 * lane + 32 - __clz(zeros)) : 0u) - 1;
    if (lane < NWT && w.m) {
        w.m[lane] = Mt;
        w.s[lane] = St;
        w.e[lane] = Et;
        w.mb[lane] = (int)(excl & 0xffffu);
        w.sb[lane] = (int)(excl >> 16);
        w.ls[lane] = ls;
    }
    if (lane < NWT && rowtab) {
        // marked sample of each stage row: row mb + j holds the j-th marked bit
        uint32_t mm = Mt;
        int r = (int)(excl & 0xffffu);
        while (mm) {
            const int bit = __ffs(mm) - 1;
            mm &= mm - 1u;
            rowtab[r++] = (int16_t)(32 * lane + bit);
        }
    }
    Agg agg;
    agg.m = tot & 0xffffu;
    agg.s = tot >> 16;
    agg.tr = nt - 1 - lz;
    agg.full = (lz < 0) && m_prev;
    agg.poison = 0;
    return agg;
}

// The tile's aggregate alone (the count pass needs no per-word prefixes): the
// same totals as words_from_marks - marked samples, island starts, trailing
// run - from three warp reductions.
template <int TW>
__device__ __forceinline__ Agg agg_from_marks(uint32_t Mt, uint32_t m_prev, int nt, int lane)
{
    constexpr int NWT = TW / 32;
    if (lane >= NWT) Mt = 0u;
    uint32_t below = __shfl_up_sync(kFull, Mt, 1);
    if (lane == 0) below = m_prev << 31;
    const uint32_t St = Mt & ~((Mt << 1) | (below >> 31));
    const unsigned m = __reduce_add_sync(kFull, (unsigned)__popc(Mt));
    const unsigned st = __reduce_add_sync(kFull, (unsigned)__popc(St));
    const uint32_t zeros = ~Mt & range_mask(32ll * lane, 0, nt);
    const int lz = (int)__reduce_max_sync(kFull, zeros ? (unsigned)(32 * lane + 32 - __clz(zeros)) : 0u) - 1;
    Agg agg;
    agg.m = m;
    agg.s = st;
    agg.tr = nt - 1 - lz;
    agg.full = (lz < 0) && m_prev;
    agg.poison = 0;
    return agg;
}

// Marks of the tile proper from the threshold bits of the extended tile (one
// warp): returns this lane's marks word of the tile proper and, through
// *edges, bit 0 = mark of sample t0 - 1 and bit 1 = mark of sample t0 + TW.
template <int TW>
__device__ __forceinline__ uint32_t tile_marks(const KArgs &a, const TileInfo &T, const uint8_t *abyte,
                                               unsigned *edges, int lane)
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
    *edges = m_prev | (m_next << 1);
    return Mt;
}

// --------------------------------------------------------------------------- windows + merge (one warp)
// Marks, island starts and ends, prefix counts and the aggregate of one tile.
template <int TW>
__device__ __forceinline__ Agg tile_bits(const KArgs &a, const TileInfo &T, const uint8_t *abyte, TileWords w,
                                         int16_t *rowtab, int lane)
{
    unsigned edges;
    const uint32_t Mt = tile_marks<TW>(a, T, abyte, &edges, lane);
    return words_from_marks<TW>(Mt, edges & 1u, edges >> 1, (int)(T.t_end - T.t0), w, rowtab, lane);
}

// --------------------------------------------------------------------------- cross-tile scan
__device__ __forceinline__ void publish(TileStatus *st, long long tile, bool inclusive, const Agg &v,
                                        bool relaxed = false)
{
    const unsigned long long kind = inclusive ? (v.poison ? kKindPoison : kKindInc) : kKindAgg;
    const unsigned long long lo = ((unsigned long long)v.m << 2) | kind;
    const unsigned long long hi = ((unsigned long long)v.s << 33) | ((unsigned long long)v.tr << 3) |
                                  ((unsigned long long)(v.full != 0) << 2) | kind;
    // the word is the whole message (readers use nothing else on its account),
    // so a relaxed store suffices; release also waits for the thread's earlier
    // stores and atomics
    if (relaxed) st_relaxed_b128(&st[tile], lo, hi);
    else st_release_b128(&st[tile], lo, hi);
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
// Bounded: gives up after a.wait_ns or once another CTA has flagged a
// timeout, returning a poisoned prefix.
__device__ Agg look_back_in(const KArgs &a, const TileStatus *st, long long tile, int lane, unsigned *stats = nullptr)
{
    constexpr int PER = 4, BIG = 1 << 20;
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
            {  // the clock every poll (a short limit must bite); the flag every 16th
                int give_up = lane == 0 && (global_ns() - t_start > a.wait_ns || ((iter & 15u) == 15u && aborted(a)));
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

__device__ __forceinline__ Agg look_back(const KArgs &a, long long tile, int lane, unsigned *stats = nullptr)
{
    return look_back_in(a, a.status, tile, lane, stats);
}

// --------------------------------------------------------------------------- pool rows to global
// The stage area holds every sample row of the tile (row = sample - t0, pitch
// srow bytes).  Output row r of the tile is stage row rowtab[r].  Output goes
// to global rows [excl.m, excl.m + agg.m): whole 16-byte chunks from one
// thread each, the unaligned ends in smaller stores.
__device__ __forceinline__ void copy_out(const KArgs &a, const unsigned char *stage, const int16_t *rowtab,
                                         const Agg &excl, const Agg &agg, int gt, int nthr, int max_rows)
{
    long long rows = agg.m;
    if ((a.flags & DAQ_DEBUG_CHECKS) && (excl.m < 0 || rows < 0 || rows > max_rows)) {
        if (gt == 0) set_status_bit(a, DAQ_DEV_BAD_INDEX);  // more rows than the stage holds
        return;
    }
    if (excl.m + rows > a.pool_cap) {
        rows = a.pool_cap - excl.m;
        if (gt == 0) set_status_bit(a, DAQ_DEV_POOL_OVERFLOW);
    }
    if (rows <= 0) return;
    if (a.n_xtal & 1) {
        // odd crystal count: rows are not whole words; one int16 at a time
        const int X = a.n_xtal, sp = a.srow >> 1;
        const int16_t *s16 = reinterpret_cast<const int16_t *>(stage);
        int16_t *g16 = a.pool + excl.m * X;
        for (long long e = gt; e < rows * X; e += nthr) {
            const int r = (int)(e / X), x = (int)(e - (long long)r * X);
            g16[e] = s16[rowtab[r] * sp + x];
        }
        return;
    }
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(stage);
    const int P = a.srow >> 2, wpr = a.wpr;
    const long long G0 = excl.m * wpr;  // global word of the tile's first output word
    const long long n_words = rows * wpr;
    uint32_t *g32 = reinterpret_cast<uint32_t *>(a.pool) + G0;
    auto row_of = [&](uint32_t w) {
        uint32_t r = (uint32_t)(((unsigned long long)w * a.wpr_mul) >> 32);
        if (r * (uint32_t)wpr > w) --r;
        return r;
    };
    auto src_word = [&](uint32_t w) {
        const uint32_t r = row_of(w);
        return (uint32_t)rowtab[r] * (uint32_t)P + (w - r * (uint32_t)wpr);
    };
    const int head = (int)min((long long)((4 - (G0 & 3)) & 3), n_words);
    const long long n_chunks = (n_words - head) >> 2;
    const long long tail0 = head + 4 * n_chunks;
    const int n_tail = (int)(n_words - tail0);
    if (gt < head) g32[gt] = sw[src_word((uint32_t)gt)];
    else if (gt >= 4 && gt < 4 + n_tail) g32[tail0 + gt - 4] = sw[src_word((uint32_t)(tail0 + gt - 4))];
    constexpr int U = 4;
    for (long long c0 = gt; c0 < n_chunks; c0 += (long long)U * nthr) {
        uint4 out[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long c = c0 + (long long)u * nthr;
            out[u] = make_uint4(0u, 0u, 0u, 0u);
            if (c < n_chunks) {
                const uint32_t w = (uint32_t)(head + 4 * c);
                uint32_t r = row_of(w);
                uint32_t k = w - r * (uint32_t)wpr;
                uint32_t base = (uint32_t)rowtab[r] * (uint32_t)P;
                uint32_t vals[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    vals[e] = sw[base + k];
                    if (++k == (uint32_t)wpr && e < 3) {
                        k = 0;
                        ++r;
                        base = (uint32_t)rowtab[r] * (uint32_t)P;
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
        if ((a.flags & DAQ_DEBUG_CHECKS) &&
            !(idx >= 0 && T.f >= 0 && T.f < a.n_fills && T.c >= 0 && T.c < a.n_calo && start >= 0 && ilen >= 1 &&
              t_e < T.len && row_end - ilen + 1 >= 0 && row_end - ilen + 1 <= row_end)) {
            set_status_bit(a, DAQ_DEV_BAD_INDEX);  // the record would not describe the fill: skip it
            continue;
        }
        if (idx < a.hdr_cap) {
            daq_island *h = a.hdr + idx;
            h->fill = a.fill_base + T.f;
            h->calo = a.calo_base + T.c;
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
            reinterpret_cast<unsigned long long *>(a.q + a.qoff[d] + (long long)(a.calo_base + T.c) * a.qbins[d]);
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
            if ((a.flags & DAQ_DEBUG_CHECKS) &&
                !(k >= 0 && k < a.qbins[d] && a.calo_base + T.c >= 0 && a.calo_base + T.c < a.q_calos)) {
                set_status_bit(a, DAQ_DEV_BAD_INDEX);
                continue;
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
