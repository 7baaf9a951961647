// Lossless packing of pool rows on the GPU (Sec. 3: the frontend compresses
// island data losslessly before event building).  Stream format:
//   header   u32 magic 0x50514144, u32 n_xtal, u64 rows
//   offsets  u64[n_blocks + 1], n_blocks = ceil(rows / 32): byte offset of each
//            block's payload from the payload start (the last = payload size)
//   payload  block b = rows [32b, 32b + 32), the last block padded with copies
//            of the final row; per crystal x, with v_i the sample of row i:
//            z_0 = 0, z_i = zigzag(v_i - v_{i-1}) (2d for d >= 0, -2d - 1 else),
//            w = bit length of max z_i (0..17); words: (uint16)v_0 | w << 16,
//            then w bit planes, bit i of plane k = bit k of z_i.
// Consecutive pool rows are consecutive samples of an island, so the row to
// row differences of a crystal are small (noise, pulse edges) and a block's
// crystal column typically needs a few bits per sample instead of 16.
//
// One warp per block at a time, blocks b, b + W, ... (W warps in the grid).
// Each warp keeps two block buffers in shared memory: while it works on one,
// a bulk copy (one instruction, completing on the buffer's mbarrier) brings
// in its next block, so the global load latency overlaps the work.  The size
// pass puts lanes on crystal columns: a lane walks its
// column down the 32 rows OR-ing the zigzag differences (the bit length of the
// OR is that of the maximum: the column's width) and the block's size
// follows.  An exclusive scan of the block sizes (three kernels) gives the
// offsets.  The write pass puts lanes on rows (row pitch an odd number of
// words, so a warp reading one crystal down 32 rows hits 32 banks): one
// shuffle forms a column's differences and one 32 x 32 bit transpose across
// the warp turns them into bit planes held by lanes in stream order, shared
// by two or four columns when their widths allow.  The decoder is the same
// walk backwards (one load of the columns' words, the transpose, the
// differences summed by an inclusive warp scan).  (One ballot per plane, the
// first form, took 2.7x as long: the integer pipe ran out.  A single pass
// whose warps found their block's place by decoupled look-back was slower
// still: with thousands of one-block warps in flight the nearest published
// prefix lies hundreds of blocks back.)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "daq.h"
#include "daq_device.cuh"

namespace daq_pack {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kMaxX = 64;
constexpr uint32_t kMagic = 0x50514144u;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kThreads * kScanPer;
constexpr uint64_t kWaitNs = 4000000000ull;  // a block copy not landed after this: give up (error word)

__device__ __forceinline__ uint32_t zigzag(int32_t d) { return ((uint32_t)d << 1) ^ (uint32_t)(d >> 31); }

__device__ __forceinline__ int32_t unzigzag(uint32_t z) { return (z & 1u) ? -(int32_t)((z + 1u) >> 1) : (int32_t)(z >> 1); }

// Per 16-bit half, modulo 2^16: v - p (no borrow crosses the halves).
__device__ __forceinline__ uint32_t sub16x2(uint32_t v, uint32_t p)
{
    return ((v | 0x80008000u) - (p & 0x7fff7fffu)) ^ ((v ^ ~p) & 0x80008000u);
}

// Per 16-bit half: zigzag(d) = 2d for d >= 0, -2d - 1 else, i.e. (d << 1) ^
// (the half's sign spread over it); the sign comes from a byte permute that
// replicates the top bit of bytes 1 and 3.
__device__ __forceinline__ uint32_t zigzag16x2(uint32_t d)
{
    uint32_t sgn;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(sgn) : "r"(d), "r"(0u), "r"(0xbb99u));
    return ((d << 1) & 0xfffefffeu) ^ sgn;
}

// A warp's shared rows: the block's 32 rows back to back (row pitch X), as in
// the pool.  Reading one crystal down the rows strides X int16 per lane, which
// is conflict-free whenever X/2 is odd (54 crystals: 27 words per row).
constexpr int kBlockElems = 32 * kMaxX;

// Copy block b's rows (16-byte vectors; the pool and every block start are
// 16-byte aligned) into the warp's shared rows, rows past the pool's end
// repeating its final row.  Returns the number of real rows.
__device__ __forceinline__ int load_block(const int16_t *pool, long long rows, int X, long long b, int16_t *sm,
                                          int lane)
{
    const long long r0 = 32ll * b;
    const int nv = (int)min(32ll, rows - r0);
    const int n = nv * X;  // int16 elements
    const int16_t *src = pool + r0 * X;
    const int nvec = n >> 3;
    for (int k = lane; k < nvec; k += 32) reinterpret_cast<int4 *>(sm)[k] = reinterpret_cast<const int4 *>(src)[k];
    for (int e = (nvec << 3) + lane; e < n; e += 32) sm[e] = src[e];
    __syncwarp();
    for (int e = n + lane; e < 32 * X; e += 32) sm[e] = sm[(nv - 1) * X + (e - n) % X];
    __syncwarp();
    return nv;
}

// Per-warp pipeline of 32-row blocks in dynamic shared memory: two buffers
// of 64 X bytes (a block's rows back to back, row pitch X, as in the pool:
// reading one crystal down the rows strides X int16 per lane, conflict-free
// whenever X/2 is odd, as for 54 crystals), then `extra` bytes of the
// caller's, then two mbarriers.  Blocks below nfull (32 real rows) come in by
// bulk copy, one block ahead; the last block, when it is shorter, is copied by
// the lanes with its padding rows.  `wait` returns false when a copy did not
// land within kWaitNs; `drain` waits (bounded) for copies still in flight, so
// that the warp may leave.
struct BlockPipe {
    unsigned char *base, *extra;
    uint64_t *bar;
    int bufb;               // bytes of one buffer (64 X)
    uint32_t pend = 0;      // lane 0: buffers with a copy issued and not waited for
    uint32_t par = 0;       // lane 0: bit s = phase parity of buffer s's pending copy
    uint32_t next_par = 0;  // bit s = phase parity the next wait on buffer s expects

    static __host__ __device__ size_t bytes(int X, int extra) { return 2 * 64 * (size_t)X + (size_t)extra + 16; }

    __device__ BlockPipe(unsigned char *b, int X, int extra_bytes, int lane)
        : base(b), extra(b + 128 * X), bar(reinterpret_cast<uint64_t *>(b + 128 * X + extra_bytes)), bufb(64 * X)
    {
        if (lane == 0) {
            daq::mbar_init(bar, 1);
            daq::mbar_init(bar + 1, 1);
            daq::fence_mbar_init();
        }
        __syncwarp();
    }
    __device__ int16_t *buf(int s) const { return reinterpret_cast<int16_t *>(base + s * bufb); }
    // lane 0: start the copy of full block b into buffer s (the warp is done with it)
    __device__ void issue(const int16_t *pool, int X, long long b, int s)
    {
        daq::fence_proxy_async_smem();
        daq::mbar_arrive_expect_tx(bar + s, (uint32_t)bufb);
        daq::bulk_g2s(buf(s), pool + 32ll * b * X, (uint32_t)bufb, bar + s);
        pend |= 1u << s;
        par = (par & ~(1u << s)) | (next_par & (1u << s));
    }
    // every lane: block b's rows are in buffer s
    __device__ bool wait(const int16_t *pool, long long rows, int X, long long b, long long nfull, int s, int lane)
    {
        if (b < nfull) {
            if (!daq::mbar_wait_bounded(bar + s, (next_par >> s) & 1u, kWaitNs)) return false;
            next_par ^= 1u << s;
            pend &= ~(1u << s);
        } else {
            load_block(pool, rows, X, b, buf(s), lane);
        }
        return true;
    }
    // lane 0: wait (bounded) for copies still in flight, so that the warp may leave
    __device__ void drain()
    {
        for (int s = 0; s < 2; ++s)
            if (pend & (1u << s)) daq::mbar_wait_bounded(bar + s, (par >> s) & 1u, kWaitNs);
    }
};

// Block sizes, and the width of every crystal column (widths[b][x]).  Lanes
// take crystal columns here: lane x walks its column down the block's 32 rows
// (consecutive lanes read consecutive samples of a row: no bank conflict),
// OR-ing the zigzag differences in a register, so a column costs a few
// instructions per row shared by 32 columns instead of a shuffle and a
// reduction of its own.
__global__ void __launch_bounds__(kThreads) pack_size_kernel(const int16_t *pool, long long rows, int X,
                                                             long long nb, unsigned long long *sizes,
                                                             uint8_t *widths, int *perr)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BlockPipe pipe(dsm + warp * BlockPipe::bytes(X, 0), X, 0, lane);
    const long long nfull = rows / 32, W = (long long)gridDim.x * kWarps;
    long long b = (long long)blockIdx.x * kWarps + warp;
    if (lane == 0 && b < nfull) pipe.issue(pool, X, b, 0);
    for (int it = 0; b < nb; b += W, ++it) {
        const int s = it & 1;
        if (lane == 0 && b + W < nfull) pipe.issue(pool, X, b + W, s ^ 1);
        if (!pipe.wait(pool, rows, X, b, nfull, s, lane)) {
            if (lane == 0) atomicOr(perr, 1);
            break;
        }
        const int16_t *sm = pipe.buf(s);
        unsigned words = 0;
        for (int x = lane; x < X; x += 32) {
            const int16_t *col = sm + x;
            int32_t prev = col[0];
            uint32_t acc = 0;
#pragma unroll
            for (int r = 1; r < 32; ++r) {
                const int32_t v = col[r * X];
                acc |= zigzag(v - prev);
                prev = v;
            }
            const int w = 32 - __clz(acc);  // 0 for acc = 0
            widths[b * X + x] = (uint8_t)w;
            words += 1u + (unsigned)w;
        }
        words = __reduce_add_sync(kFull, words);
        if (lane == 0) sizes[b] = 4ull * words;
        __syncwarp();
    }
    if (lane == 0) pipe.drain();
}

// ------------------------------------------------------------------ exclusive scan of the block sizes
__global__ void __launch_bounds__(kThreads) scan_reduce_kernel(const unsigned long long *v, long long n,
                                                               unsigned long long *chunk)
{
    __shared__ unsigned long long s[kWarps];
    const long long base = (long long)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    unsigned long long t = 0;
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) t += v[base + i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(kFull, t, d);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0;
        for (int w = 0; w < kWarps; ++w) a += s[w];
        chunk[blockIdx.x] = a;
    }
}

// One block: chunk sums -> exclusive prefixes (in place); chunk[n_chunks] = total.
__global__ void __launch_bounds__(1024) scan_top_kernel(unsigned long long *chunk, long long n_chunks)
{
    __shared__ unsigned long long s[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long base = 0; base < n_chunks; base += 1024) {
        const long long i = base + threadIdx.x;
        const unsigned long long v = i < n_chunks ? chunk[i] : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) s[warp] = x;
        __syncthreads();
        unsigned long long pre = carry;
        for (int w = 0; w < warp; ++w) pre += s[w];
        if (i < n_chunks) chunk[i] = pre + x - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = pre + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) chunk[n_chunks] = carry;
}

// offsets[b] = exclusive prefix (workspace, and the stream's table when it
// fits), offsets[nb] = payload size, *out_bytes = whole stream size.
__global__ void __launch_bounds__(kThreads) scan_apply_kernel(const unsigned long long *v, long long n,
                                                              const unsigned long long *chunk,
                                                              unsigned long long *offs, unsigned char *out,
                                                              long long cap, long long *out_bytes, const int *perr)
{
    __shared__ unsigned long long s[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    unsigned long long loc[kScanPer], t = 0;
    for (int i = 0; i < kScanPer; ++i) {
        loc[i] = base + i < n ? v[base + i] : 0ull;
        t += loc[i];
    }
    unsigned long long x = t;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s[warp] = x;
    __syncthreads();
    unsigned long long pre = chunk[blockIdx.x];
    for (int w = 0; w < warp; ++w) pre += s[w];
    pre += x - t;
    const long long table = 16;  // the offsets table starts after the 16-byte header
    for (int i = 0; i < kScanPer; ++i) {
        const long long k = base + i;  // entries 0..n (entry n: the payload size)
        if (k <= n) {
            offs[k] = pre;
            if (table + 8 * k + 8 <= cap) reinterpret_cast<unsigned long long *>(out + table)[k] = pre;
            if (k == n) *out_bytes = *perr ? -1 : 16 + 8 * (n + 1) + (long long)pre;  // -1: the size pass gave up
        }
        pre += loc[i];
    }
}

// 32 x 32 bit transpose across the warp: lane j receives bit j of every lane's
// x (bit i of the result = bit j of lane i's x).  Five stages of the recursive
// block swap: at stage s the lane pairs (l, l ^ s) exchange the off-diagonal
// s x s blocks - the lane with bit s clear keeps the bits whose index has bit
// s clear (mask m) and takes its partner's such bits shifted up by s, the
// other keeps ~m and takes its partner's ~m bits shifted down by s.  Each
// shift is a rotation (funnel shift) whose unwanted bits the select drops, so
// a stage is one shuffle, one rotation and one bitwise select.
struct Transpose {
    uint32_t keep[5];
    int rot[5];
    __device__ __forceinline__ explicit Transpose(int lane)
    {
        constexpr uint32_t kMask[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            const int sft = 16 >> t;
            const bool low = (lane & sft) == 0;
            keep[t] = low ? kMask[t] : ~kMask[t];
            rot[t] = low ? sft : 32 - sft;
        }
    }
    __device__ __forceinline__ uint32_t operator()(uint32_t x) const
    {
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            const uint32_t y = __shfl_xor_sync(kFull, x, 16 >> t);
            const uint32_t r = __funnelshift_l(y, y, rot[t]);
            x = (x & keep[t]) | (r & ~keep[t]);
        }
        return x;
    }
    // two independent transposes, stage by stage (their shuffles overlap)
    __device__ __forceinline__ void two(uint32_t &x, uint32_t &z) const
    {
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            const uint32_t y = __shfl_xor_sync(kFull, x, 16 >> t);
            const uint32_t w = __shfl_xor_sync(kFull, z, 16 >> t);
            x = (x & keep[t]) | (__funnelshift_l(y, y, rot[t]) & ~keep[t]);
            z = (z & keep[t]) | (__funnelshift_l(w, w, rot[t]) & ~keep[t]);
        }
    }
};

// Crystal columns go through the transpose four at a time when all four
// widths are <= 7 (the common case for noise-dominated island rows), else in
// pairs when both are <= 15, else alone.  A group of G = 8, 16 or 32 lanes
// serves one column: its z << 1 sits at bit G g of the transposed word, so
// lane G g + k + 1 receives plane k and the group's first lane, which receives
// zeros, carries the head word instead.  One store then writes every column's
// words, which lie back to back: the head, then the planes.
// - Four: byte g of (w4 + 0x01010101) * 0x01010100 is the words of the columns
//   before g (w4 = the four widths as bytes); lane 0 broadcasts the first
//   samples two to a word.
// - Alone (a width of 16 or 17: a difference of at least 2^14).
// kPairs (even X): in the four-column path a lane reads its row's crystals two
// to a 32-bit word and forms both differences and zigzag codes at once, in
// 16-bit halves (exact there: every difference is within +-64).
// A block copy that does not land within kWaitNs sets *out_bytes to -1.
template <bool kPairs>
__global__ void __launch_bounds__(kThreads, 4) pack_write_kernel(const int16_t *pool, long long rows, int X, long long nb,
                                                              const unsigned long long *offs, const uint8_t *widths,
                                                              unsigned char *out, long long cap, long long *out_bytes)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BlockPipe pipe(dsm + warp * BlockPipe::bytes(X, kMaxX), X, kMaxX, lane);
    uint8_t *wsm = pipe.extra;  // widths of the block being written
    const Transpose transpose(lane);
    const int k16 = lane & 15, k8 = lane & 7;
    const bool hi16 = lane >= 16;
    const int g4 = lane >> 3, g8 = 8 * g4;  // four-column group of this lane, its byte
    uint32_t *out32 = reinterpret_cast<uint32_t *>(out);
    const long long head = 16 + 8 * (nb + 1);
    if (blockIdx.x == 0 && threadIdx.x == 0 && cap >= 16) {
        out32[0] = kMagic;
        out32[1] = (uint32_t)X;
        reinterpret_cast<unsigned long long *>(out)[1] = (unsigned long long)rows;
    }
    const long long nfull = rows / 32, Wn = (long long)gridDim.x * kWarps;
    long long b = (long long)blockIdx.x * kWarps + warp;
    int w_lo = 0, w_hi = 0;  // widths of columns lane and lane + 32 of the block to come
    auto widths_of = [&](long long bb) {
        w_lo = lane < X ? widths[bb * X + lane] : 0;
        w_hi = lane + 32 < X ? widths[bb * X + lane + 32] : 0;
    };
    if (b < nb) {
        if (lane == 0 && b < nfull) pipe.issue(pool, X, b, 0);
        widths_of(b);
    }
    for (int it = 0; b < nb; b += Wn, ++it) {
        const int s = it & 1;
        if (lane < X) wsm[lane] = (uint8_t)w_lo;
        if (lane + 32 < X) wsm[lane + 32] = (uint8_t)w_hi;
        if (b + Wn < nb) {
            if (lane == 0 && b + Wn < nfull) pipe.issue(pool, X, b + Wn, s ^ 1);
            widths_of(b + Wn);
        }
        if (!pipe.wait(pool, rows, X, b, nfull, s, lane)) {
            if (lane == 0) *out_bytes = -1;
            break;
        }
        __syncwarp();
        const int16_t *row = pipe.buf(s) + lane * X;
        const long long start = head + (long long)offs[b];  // bytes, a multiple of 4
        uint32_t *dst = out32 + (start >> 2);
        // words that may be written from the block's start (a block is < 2^11 words)
        const int room = (int)(max(0ll, min(cap - start, 1ll << 20)) >> 2);
        int o = 0;  // words of the block written so far
        auto single = [&](int x) {
            const int32_t v = row[x];
            const uint32_t z = zigzag(v - __shfl_up_sync(kFull, v, 1));
            const int w = wsm[x];
            const uint32_t planes = transpose(z << 1);
            const uint32_t word = lane ? planes : ((uint32_t)(uint16_t)v | ((uint32_t)w << 16));
            if (lane <= w && o + lane < room) dst[o + lane] = word;
            o += 1 + w;
        };
        auto pair = [&](int x) {
            const int wa = wsm[x], wb = wsm[x + 1];
            if (max(wa, wb) > 15) {
                single(x);
                single(x + 1);
                return;
            }
            const int32_t va = row[x], vb = row[x + 1];
            const uint32_t za = zigzag(va - __shfl_up_sync(kFull, va, 1));
            const uint32_t zb = zigzag(vb - __shfl_up_sync(kFull, vb, 1));
            const uint32_t planes = transpose((za << 1) | (zb << 17));
            const uint32_t firsts = __shfl_sync(kFull, (uint32_t)(uint16_t)va | ((uint32_t)vb << 16), 0);
            const int w = hi16 ? wb : wa;
            const uint32_t hw = (hi16 ? firsts >> 16 : firsts & 0xffffu) | ((uint32_t)w << 16);
            const int i = o + (hi16 ? 1 + wa : 0) + k16;
            if (k16 <= w && i < room) dst[i] = k16 ? planes : hw;
            o += 2 + wa + wb;
        };
        // four columns of width <= 7: their z << 1 as bytes, lane 0's samples two to a word
        auto quad_z = [&](int x, uint32_t &zq, uint32_t &f01, uint32_t &f23) {
            if constexpr (kPairs) {
                const uint32_t *row32 = reinterpret_cast<const uint32_t *>(row);
                const uint32_t v01 = row32[x >> 1], v23 = row32[(x >> 1) + 1];
                const uint32_t z01 = zigzag16x2(sub16x2(v01, __shfl_up_sync(kFull, v01, 1)));
                const uint32_t z23 = zigzag16x2(sub16x2(v23, __shfl_up_sync(kFull, v23, 1)));
                zq = __byte_perm(z01, z23, 0x6420) << 1;  // z < 128: no bit crosses into the next byte
                f01 = __shfl_sync(kFull, v01, 0);
                f23 = __shfl_sync(kFull, v23, 0);
            } else {
                const int32_t v0 = row[x], v1 = row[x + 1], v2 = row[x + 2], v3 = row[x + 3];
                const uint32_t z0 = zigzag(v0 - __shfl_up_sync(kFull, v0, 1));
                const uint32_t z1 = zigzag(v1 - __shfl_up_sync(kFull, v1, 1));
                const uint32_t z2 = zigzag(v2 - __shfl_up_sync(kFull, v2, 1));
                const uint32_t z3 = zigzag(v3 - __shfl_up_sync(kFull, v3, 1));
                zq = (z0 << 1) | (z1 << 9) | (z2 << 17) | (z3 << 25);
                f01 = __shfl_sync(kFull, (uint32_t)(uint16_t)v0 | ((uint32_t)v1 << 16), 0);
                f23 = __shfl_sync(kFull, (uint32_t)(uint16_t)v2 | ((uint32_t)v3 << 16), 0);
            }
        };
        // store the words of four columns (widths w4 as bytes) from their transposed planes
        auto quad_store = [&](uint32_t planes, uint32_t w4, uint32_t f01, uint32_t f23) {
            const uint32_t fp = g4 < 2 ? f01 : f23;
            const uint32_t w = (w4 >> g8) & 0xffu;
            const uint32_t hw = ((g4 & 1) ? fp >> 16 : fp & 0xffffu) | (w << 16);
            const uint32_t before = (w4 + 0x01010101u) * 0x01010100u;  // byte g: words of columns < g
            const int i = o + (int)((before >> g8) & 0xffu) + k8;
            if (k8 <= (int)w && i < room) dst[i] = k8 ? planes : hw;
            o += (int)(before >> 24) + 1 + (int)(w4 >> 24);
        };
        auto narrow = [](uint32_t w4) { return ((w4 + 0x78787878u) & 0x80808080u) == 0u; };  // every width <= 7
        auto group = [&](int x, uint32_t w4) {
            if (!narrow(w4)) {
                pair(x);
                pair(x + 2);
                return;
            }
            uint32_t zq, f01, f23;
            quad_z(x, zq, f01, f23);
            quad_store(transpose(zq), w4, f01, f23);
        };
        int x = 0;
        for (; x + 7 < X; x += 8) {  // two groups of four: both narrow, their transposes overlap
            const uint32_t w4a = *reinterpret_cast<const uint32_t *>(wsm + x);
            const uint32_t w4b = *reinterpret_cast<const uint32_t *>(wsm + x + 4);
            if (narrow(w4a) && narrow(w4b)) {
                uint32_t za, fa01, fa23, zb, fb01, fb23;
                quad_z(x, za, fa01, fa23);
                quad_z(x + 4, zb, fb01, fb23);
                transpose.two(za, zb);
                quad_store(za, w4a, fa01, fa23);
                quad_store(zb, w4b, fb01, fb23);
            } else {
                group(x, w4a);
                group(x + 4, w4b);
            }
        }
        for (; x + 3 < X; x += 4) group(x, *reinterpret_cast<const uint32_t *>(wsm + x));
        for (; x + 1 < X; x += 2) pair(x);
        if (x < X) single(x);
        __syncwarp();
    }
    if (lane == 0) pipe.drain();
}

__global__ void __launch_bounds__(kThreads) unpack_kernel(const unsigned char *in, long long in_bytes, long long rows,
                                                          int X, long long nb, int16_t *pool_out, int *err)
{
    __shared__ __align__(16) int16_t sm_all[kWarps][kBlockElems];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int16_t *sm = sm_all[warp];
    const int P = X;
    const Transpose transpose(lane);
    const long long head = 16 + 8 * (nb + 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t *h = reinterpret_cast<const uint32_t *>(in);
        if (h[0] != kMagic || h[1] != (uint32_t)X || reinterpret_cast<const unsigned long long *>(in)[1] !=
                                                             (unsigned long long)rows)
            atomicOr(err, 1);
    }
    const unsigned long long *offs = reinterpret_cast<const unsigned long long *>(in + 16);
    for (long long b = (long long)blockIdx.x * kWarps + warp; b < nb; b += (long long)gridDim.x * kWarps) {
        if (head > in_bytes) {  // the offsets table itself is cut short
            if (lane == 0) atomicOr(err, 2);
            continue;
        }
        const unsigned long long off = offs[b];
        bool bad = off > (unsigned long long)(in_bytes - head) || (off & 3ull);
        long long pos = head + (long long)(bad ? 0ull : off);  // bytes read so far end at pos
        for (int x = 0; x < X && !bad;) {
            // the next 32 words: up to four columns' head words and planes
            const uint32_t *p = reinterpret_cast<const uint32_t *>(in + pos);
            const uint32_t q = pos + 4ll * lane + 4 <= in_bytes ? p[lane] : 0u;
            const uint32_t h0 = __shfl_sync(kFull, q, 0);
            const int w0 = (int)(h0 >> 16);
            // four columns of width <= 7 at once: their head words lie at 0, i1, i2, i3
            const int i1 = 1 + min(w0, 8);
            const uint32_t h1 = __shfl_sync(kFull, q, i1);
            const int w1 = (int)(h1 >> 16), i2 = i1 + 1 + min(w1, 8);
            const uint32_t h2 = __shfl_sync(kFull, q, i2);
            const int w2 = (int)(h2 >> 16), i3 = i2 + 1 + min(w2, 8);
            const uint32_t h3 = __shfl_sync(kFull, q, i3);
            const int w3 = (int)(h3 >> 16), total = i3 + 1 + min(w3, 8);
            if (x + 3 < X && max(max(w0, w1), max(w2, w3)) <= 7 && pos + 4ll * total <= in_bytes) {
                // lane 8g + k + 1 takes plane k of column g: the transpose gives lane i
                // bit k of z_{g,i} at bit 8g + k + 1
                const int g = lane >> 3, k = lane & 7;
                const int ig = g == 0 ? 0 : g == 1 ? i1 : g == 2 ? i2 : i3;
                const int wg = g == 0 ? w0 : g == 1 ? w1 : g == 2 ? w2 : w3;
                const uint32_t pl = __shfl_sync(kFull, q, (ig + k) & 31);
                const uint32_t t = transpose(k >= 1 && k <= wg ? pl : 0u);
                // |difference| <= 64, so 32 of them sum below 2^15: two columns share a scan
                int32_t d01 = lane ? unzigzag((t >> 1) & 0x7fu) + unzigzag((t >> 9) & 0x7fu) * 65536 : 0;
                int32_t d23 = lane ? unzigzag((t >> 17) & 0x7fu) + unzigzag((t >> 25) & 0x7fu) * 65536 : 0;
#pragma unroll
                for (int s = 1; s < 32; s <<= 1) {
                    const int32_t y01 = __shfl_up_sync(kFull, d01, s), y23 = __shfl_up_sync(kFull, d23, s);
                    if (lane >= s) {
                        d01 += y01;
                        d23 += y23;
                    }
                }
                const int32_t s0 = (int16_t)(d01 & 0xffff), s2 = (int16_t)(d23 & 0xffff);
                const int32_t s1 = (d01 - s0) >> 16, s3 = (d23 - s2) >> 16;
                int16_t *r = sm + lane * P + x;
                r[0] = (int16_t)((int32_t)(int16_t)(h0 & 0xffffu) + s0);
                r[1] = (int16_t)((int32_t)(int16_t)(h1 & 0xffffu) + s1);
                r[2] = (int16_t)((int32_t)(int16_t)(h2 & 0xffffu) + s2);
                r[3] = (int16_t)((int32_t)(int16_t)(h3 & 0xffffu) + s3);
                pos += 4ll * total;
                x += 4;
                continue;
            }
            // one column
            if (pos + 4 > in_bytes || w0 > 17 || pos + 4ll * (1 + w0) > in_bytes) {
                bad = true;
                break;
            }
            pos += 4ll * (1 + w0);
            // lane k + 1 holds plane k: the transpose gives lane i bit k of z_i at bit k + 1
            const uint32_t z = transpose(lane >= 1 && lane <= w0 ? q : 0u) >> 1;
            int32_t d = lane ? unzigzag(z) : 0;
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, d, s);
                if (lane >= s) d += y;
            }
            sm[lane * P + x] = (int16_t)((int32_t)(int16_t)(h0 & 0xffffu) + d);
            ++x;
        }
        if (bad) {
            if (lane == 0) atomicOr(err, 2);
            continue;
        }
        __syncwarp();
        const long long r0 = 32ll * b;
        const int nv = (int)min(32ll, rows - r0);
        int16_t *dst = pool_out + r0 * X;
        const int n = nv * X;
        int done = 0;
        if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {  // 16-byte vectors where the output allows
            const int nvec = n >> 3;
            for (int k = lane; k < nvec; k += 32) reinterpret_cast<int4 *>(dst)[k] = reinterpret_cast<const int4 *>(sm)[k];
            done = nvec << 3;
        }
        for (int e = done + lane; e < n; e += 32) dst[e] = sm[e];
        __syncwarp();
    }
}

// Grid of a pipelined kernel: every CTA resident at once (its warps step
// through blocks), at most one warp per block.  The kernel's dynamic
// shared-memory limit is raised once per device to what the largest n_xtal
// needs (smem_max; a later call must never lower it), and the resident count
// is found once per (kernel slot, device, n_xtal) and kept.
constexpr int kGridDevices = 16;
int g_resident[3][kGridDevices][kMaxX + 1] = {};  // CTAs resident per GPU, 0 = not known yet
bool g_limit_set[3][kGridDevices] = {};

template <typename K> int pipelined_grid(int slot, K kernel, int X, size_t smem, size_t smem_max, long long nb)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    int resident = dev < kGridDevices ? g_resident[slot][dev][X] : 0;
    if (resident == 0) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 0;
        if (dev >= kGridDevices || !g_limit_set[slot][dev]) {
            if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) != cudaSuccess)
                return 0;
            if (dev < kGridDevices) g_limit_set[slot][dev] = true;
        }
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, smem) != cudaSuccess || per < 1)
            return 0;
        resident = per * sms;
        if (dev < kGridDevices) g_resident[slot][dev][X] = resident;
    }
    const long long want = (nb + kWarps - 1) / kWarps;
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)resident));
}

int grid_blocks(long long nb)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (nb + kWarps - 1) / kWarps;
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)std::max(sms, 1) * 16));
}

struct PackWs {
    size_t sizes, offs, chunk, widths, err, total;
};

PackWs pack_ws(long long nb, int X)
{
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    PackWs w;
    w.sizes = 0;
    w.offs = up(8 * (size_t)std::max<long long>(nb, 1));
    w.chunk = up(w.offs + 8 * (size_t)(nb + 1));
    const long long n_chunks = (nb + kScanChunk - 1) / kScanChunk;
    w.widths = up(w.chunk + 8 * (size_t)(n_chunks + 1));
    w.err = up(w.widths + (size_t)std::max<long long>(nb, 1) * (size_t)X);
    w.total = up(w.err + sizeof(int));
    return w;
}

}  // namespace daq_pack

using namespace daq_pack;

extern "C" {

int64_t daq_pack_bound(int64_t rows, int n_xtal)
{
    if (rows < 0 || n_xtal < 1 || n_xtal > kMaxX) return -1;
    const int64_t nb = (rows + 31) / 32;
    return 16 + 8 * (nb + 1) + nb * (int64_t)n_xtal * 4 * 18;
}

int daq_pack_workspace_size(int64_t rows, int n_xtal, size_t *bytes)
{
    if (!bytes || rows < 0 || n_xtal < 1 || n_xtal > kMaxX) return DAQ_EINVAL;
    *bytes = pack_ws((rows + 31) / 32, n_xtal).total;
    return DAQ_OK;
}

int daq_pack_pool(const int16_t *pool, int64_t rows, int n_xtal, void *out, int64_t out_cap, int64_t *out_bytes,
                  void *workspace, size_t workspace_bytes, void *stream)
{
    if (rows < 0 || n_xtal < 1 || out_cap < 0 || !out_bytes || (rows > 0 && !pool)) return DAQ_EINVAL;
    if (n_xtal > kMaxX) return DAQ_EUNSUPPORTED;
    if ((out_cap > 0 && !out) || (reinterpret_cast<uintptr_t>(out) & 15) || (reinterpret_cast<uintptr_t>(out_bytes) & 7) ||
        (reinterpret_cast<uintptr_t>(pool) & 15))
        return DAQ_EINVAL;
    const long long nb = (rows + 31) / 32;
    const PackWs w = pack_ws(nb, n_xtal);
    if (!workspace || workspace_bytes < w.total || (reinterpret_cast<uintptr_t>(workspace) & 15)) return DAQ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    auto *sizes = reinterpret_cast<unsigned long long *>(ws + w.sizes);
    auto *offs = reinterpret_cast<unsigned long long *>(ws + w.offs);
    auto *chunk = reinterpret_cast<unsigned long long *>(ws + w.chunk);
    auto *widths = reinterpret_cast<uint8_t *>(ws + w.widths);
    auto *perr = reinterpret_cast<int *>(ws + w.err);
    unsigned char *o = static_cast<unsigned char *>(out);
    const long long n_apply = nb / kScanChunk + 1;  // blocks covering entries 0..nb
    const size_t smem_size = kWarps * BlockPipe::bytes(n_xtal, 0);
    const size_t smem_write = kWarps * BlockPipe::bytes(n_xtal, kMaxX);
    const bool pairs = (n_xtal % 2) == 0;
    const auto write_kernel = pairs ? pack_write_kernel<true> : pack_write_kernel<false>;
    const size_t max_size = kWarps * BlockPipe::bytes(kMaxX, 0), max_write = kWarps * BlockPipe::bytes(kMaxX, kMaxX);
    const int g_size = nb > 0 ? pipelined_grid(0, pack_size_kernel, n_xtal, smem_size, max_size, nb) : 1;
    const int g_write = pipelined_grid(pairs ? 1 : 2, write_kernel, n_xtal, smem_write, max_write,
                                       std::max<long long>(nb, 1));
    if (g_size < 1 || g_write < 1) return DAQ_ECUDA;
    if (cudaMemsetAsync(perr, 0, sizeof(int), s) != cudaSuccess) return DAQ_ECUDA;
    if (nb > 0) pack_size_kernel<<<g_size, kThreads, smem_size, s>>>(pool, rows, n_xtal, nb, sizes, widths, perr);
    if (nb > 0) scan_reduce_kernel<<<(unsigned)((nb + kScanChunk - 1) / kScanChunk), kThreads, 0, s>>>(sizes, nb, chunk);
    else if (cudaMemsetAsync(chunk, 0, 8, s) != cudaSuccess) return DAQ_ECUDA;
    scan_top_kernel<<<1, 1024, 0, s>>>(chunk, nb > 0 ? (nb + kScanChunk - 1) / kScanChunk : 0);
    scan_apply_kernel<<<(unsigned)n_apply, kThreads, 0, s>>>(sizes, nb, chunk, offs, o, out_cap,
                                                             reinterpret_cast<long long *>(out_bytes), perr);
    write_kernel<<<g_write, kThreads, smem_write, s>>>(pool, rows, n_xtal, nb, offs, widths, o, out_cap,
                                                       reinterpret_cast<long long *>(out_bytes));
    return cudaGetLastError() == cudaSuccess ? DAQ_OK : DAQ_ECUDA;
}

int daq_unpack_pool(const void *in, int64_t in_bytes, int64_t rows, int n_xtal, int16_t *pool_out, int32_t *err,
                    void *stream)
{
    if (!in || in_bytes < 16 || rows < 0 || n_xtal < 1 || !err || (rows > 0 && !pool_out) ||
        (reinterpret_cast<uintptr_t>(in) & 15))
        return DAQ_EINVAL;
    if (n_xtal > kMaxX) return DAQ_EUNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(err, 0, sizeof(int32_t), s) != cudaSuccess) return DAQ_ECUDA;
    const long long nb = (rows + 31) / 32;
    unpack_kernel<<<grid_blocks(std::max<long long>(nb, 1)), kThreads, 0, s>>>(
        static_cast<const unsigned char *>(in), in_bytes, rows, n_xtal, nb, pool_out, err);
    return cudaGetLastError() == cudaSuccess ? DAQ_OK : DAQ_ECUDA;
}

}  // extern "C"
