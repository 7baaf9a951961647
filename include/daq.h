/*
 * daq.h - C ABI of the GB300 (sm_103a) muon g-2 waveform DAQ hot path.
 *
 * The library runs, on one GPU, the per-fill processing of 12-bit, 800 MSPS
 * calorimeter waveforms that W. Gohn, "Data Acquisition with GPUs: The DAQ
 * for the Muon g-2 Experiment at Fermilab" (arXiv:1611.04959), Sec. 3 and
 * Table 2, assigns to the GPU:
 *   T-method: sum the crystals of a calorimeter sample by sample, subtract
 *             pedestals, apply a threshold, add pre- and post-samples, merge
 *             overlapping windows into islands, save every crystal's raw
 *             samples over each island (Table 2 rows 1-6; Sec. 3 T-method);
 *   Q-method: decimate the pedestal-subtracted sum and accumulate it fill by
 *             fill into histograms (Table 2 rows 7-8; Sec. 3 Q-method).
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" are CUDA device (or managed) addresses on the
 *     current device; "host" pointers are ordinary host memory.
 *   - The caller owns every buffer.  daq_process_fills allocates nothing; it
 *     enqueues work on params->stream and returns without waiting, unless
 *     DAQ_SYNC is set.
 *   - Return values are daq_status codes (0 = success, negative = error).
 *     Nothing in the library aborts, traps or exits the process.
 */
#ifndef DAQ_H
#define DAQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum daq_status {
    DAQ_OK = 0,
    DAQ_EINVAL = -1,       /* bad shape, parameter, null or misaligned pointer, short workspace */
    DAQ_ECAPACITY = -2,    /* island records or pool rows did not fit; counts hold the sizes needed */
    DAQ_ECUDA = -3,        /* a CUDA call or kernel launch failed */
    DAQ_ETIMEOUT = -4,     /* a bounded device-side wait gave up; outputs are incomplete */
    DAQ_EUNSUPPORTED = -5, /* valid request this build does not handle (e.g. n_xtal > 64) */
    DAQ_ESCRATCH = -6,     /* daq_process_fills_static: the call needs more scratch than the built-in area */
    DAQ_EINDEX = -7        /* DAQ_DEBUG_CHECKS: a computed output index failed its check; that store was skipped */
};

/* params->flags */
#define DAQ_SKIP_Q 1u        /* leave qhist_inout untouched */
#define DAQ_SKIP_ISLANDS 2u  /* compute counts, write no island records, pool rows or pedestals */
#define DAQ_SYNC 4u          /* wait for the stream, then return the device-side status */
#define DAQ_PACK_POOL 8u     /* daq_process_fills_host: return the pool rows packed (see daq_pack_pool) */
#define DAQ_DEBUG_CHECKS 16u /* check every computed record, pool and Q index before its store (see below) */
#define DAQ_SPARSE 32u       /* the compact pass passes over tiles without a marked sample (see below) */

/* Bits of counts[2] (device-side status, OR-ed by the kernels). */
#define DAQ_DEV_HDR_OVERFLOW 1
#define DAQ_DEV_POOL_OVERFLOW 2
#define DAQ_DEV_TIMEOUT 4
#define DAQ_DEV_BAD_FILL_LEN 8
#define DAQ_DEV_BAD_INDEX 16 /* DAQ_DEBUG_CHECKS: an index check failed and the store was skipped */

/*
 * One island (Table 2 row 5 "save an array of identified islands"; Sec. 3:
 * the array of island data goes back to host memory).  An island is a maximal
 * run of samples [start, start + len) of one calorimeter-fill whose
 * pedestal-subtracted crystal sum crosses the threshold somewhere within
 * [t - post, t + pre] of each sample t.  Its raw samples are pool rows
 * pool_row .. pool_row + len - 1.  24 bytes, naturally aligned.
 */
typedef struct daq_island {
    int32_t fill;     /* params->fill_base + fill index within the call */
    int32_t calo;     /* calorimeter index */
    int32_t start;    /* first sample of the island */
    int32_t len;      /* number of samples */
    int64_t pool_row; /* first pool row holding the island's samples */
} daq_island;

/*
 * Parameters of one call.  Initialise with daq_params_default().
 *   threshold    T: a sample crosses when S[t] > T, S = crystal sum minus the
 *                summed pedestals (Table 2 row 2; Sec. 3 T-method).
 *   pre, post    samples added before / after every crossing (Table 2 row 3);
 *                0 <= pre, post; pre + post <= 512.
 *   ped_samples  pedestal window: the first ped_samples samples of each crystal
 *                (Table 2 row 1 uses 100); >= 1.  Each crystal's pedestal is
 *                floor((sum + floor(n/2)) / n), n = min(ped_samples, fill length).
 *   n_decim      number of Q decimation factors (0, 1 or 2); decim[i] >= 1.
 *   fill_base    added to the fill index written into island records.
 *   fill_len     device int32[n_fills] fill lengths (0 <= len <= n_samples), or
 *                NULL for n_samples each.  Out-of-range values are clamped and
 *                flagged with DAQ_DEV_BAD_FILL_LEN.
 *   flags        DAQ_SKIP_Q | DAQ_SKIP_ISLANDS | DAQ_SYNC | DAQ_DEBUG_CHECKS |
 *                DAQ_SPARSE.
 *                DAQ_DEBUG_CHECKS: before each store the kernels check the
 *                index they computed against what the call's own arithmetic
 *                allows - an island record's index, fill, calorimeter, start and
 *                length against the fill, its pool rows against the rows of the
 *                tiles before it, a tile's pool rows against the tile's width,
 *                a Q bin against the histogram's bins and calorimeter rows.  A
 *                failed check sets DAQ_DEV_BAD_INDEX and skips that store; the
 *                call then returns DAQ_EINDEX.  (Capacity shortfalls are not
 *                index errors: they stay DAQ_ECAPACITY.)  For debugging: no
 *                check fails on a correct build, and outputs are identical
 *                with and without the flag.
 *                DAQ_SPARSE (two-pass form): the compact pass takes only the
 *                tiles that hold a marked sample (a tile without one has no
 *                pool rows and starts no island), finding the next from the
 *                count records of the 32 tiles after it at once.  Outputs are
 *                identical with and without it.  Where few tiles hold islands
 *                it halves the compact pass (0.217 -> 0.117 ms on a fill with
 *                8.6% of samples in islands); where nearly all do, the extra
 *                steps cost about 0.5%.  The batch tuner tries both.
 *   tile         samples per tile: 0 = chosen by the library (two-pass form: the
 *                width of least estimated count-pass cost, 448 for the nominal
 *                windows and 384 when the halo of post + pre samples is too
 *                wide for two count CTAs per SM at 448; other forms: 448);
 *                else the largest width not above 128, 224, 384, 448 or 960
 *                that this form supports and whose shared-memory plan fits
 *                (384 only for the two-pass form, 960 only for the plain
 *                kernel).
 *   grid         0  = two-pass form (count kernel, scan, compact kernel), grids
 *                     from occupancy (default);
 *                > 0 = two-pass form with exactly this many CTAs per kernel;
 *                -1 = single-pass plain kernel, one CTA per tile;
 *                -2 = single-pass plain kernel, persistent;
 *                -3 = single-pass pipelined kernel (one CTA per SM, warp roles);
 *                -4 = single-launch form: the two passes in one cooperative
 *                     launch, the compact role a bounded distance behind the
 *                     count role so that its re-read hits L2;
 *                -5 = streaming single pass: one CTA per SM whose warps count
 *                     tiles, look back over earlier tiles' states and compact
 *                     each tile from L2 once its prefix is known (rows must be
 *                     16-byte aligned with n_samples % 8 == 0, else the call
 *                     takes the two-pass form);
 *                -6 = single-read form: one CTA per SM reads every sample from
 *                     HBM once; the crystal-sum warps write each tile's raw
 *                     rows into the SM's Tensor Memory, where they wait for the
 *                     tile's prefix, and the marked ones are then staged and
 *                     bulk-copied to the pool (the same row and n_xtal
 *                     conditions as -5, and n_xtal even, else the two-pass
 *                     form).  The kernel takes all 512 Tensor Memory columns
 *                     of each SM it runs on for its duration.
 *   stream       cudaStream_t (NULL = legacy default stream).
 *   workspace    device scratch of at least daq_workspace_size() bytes,
 *                16-byte aligned; reused by the call and not to be shared by
 *                calls that may run at the same time.
 *   events       NULL, or a host array of DAQ_N_EVENTS cudaEvent_t that the call
 *                records on `stream`: [0] start, [1] after the pedestal kernel,
 *                [2] after the count (single-pass: tile) kernel, [3] after the
 *                scan, [4] end (per-kernel timing).
 *   trace        NULL, or device uint64[max_tiles][DAQ_TRACE_WORDS] (max_tiles
 *                from daq_trace_tiles()): per-tile %globaltimer stamps of each
 *                stage (profiling only; costs a few stores per tile).
 *   calo_base    added to the calorimeter index in island records and in the
 *                Q rows the call adds to (>= 0), so that a call over a group of
 *                calorimeters of a larger array writes their true indices.
 *   lag_tiles    single-launch form (grid -4): tiles the count role may run
 *                ahead of the compact role (0 = 1024; at least 640).
 *   q_calos      calorimeters in the qhist_inout array (0 = n_calo); calo_base
 *                + n_calo must not exceed it (so calo_base > 0 needs q_calos).
 *                Calorimeter c of the call adds to row calo_base + c of each
 *                decimation's block of q_calos rows.
 *   wait_limit_ns  limit of each device-side wait on state that other CTAs
 *                publish (0 = 4 s): the look-back over earlier tiles (every
 *                form's scan), and the single-launch form's scanner and lag
 *                waits.  A wait that runs out sets DAQ_DEV_TIMEOUT; every CTA
 *                then stops taking work, waits for its own copies in flight
 *                and exits, and the call returns DAQ_ETIMEOUT with incomplete
 *                outputs.  The next call starts clean.  Waits of a CTA on its
 *                own warps keep the 4 s limit.
 */
typedef struct daq_params {
    int32_t threshold;
    int32_t pre;
    int32_t post;
    int32_t ped_samples;
    int32_t n_decim;
    int32_t decim[2];
    int32_t fill_base;
    const int32_t *fill_len;
    uint32_t flags;
    int32_t tile;
    int32_t grid;
    int32_t calo_base;
    void *stream;
    void *workspace;
    size_t workspace_bytes;
    void *const *events;
    uint64_t *trace;
    int32_t q_calos;
    int32_t lag_tiles;
    uint64_t wait_limit_ns;
} daq_params;

#define DAQ_N_EVENTS 5

/* Per-tile trace record: stamps in nanoseconds (%globaltimer), 0 = stage not reached.
 * [0] ticket taken  [1] load issued  [2] load landed  [3] sums done  [4] marks done
 * [5] look-back start  [6] prefix known  [7] rows staged  [8] writer start
 * [9] rows written  [10] SM id  [11] tile width  [12] copy start  [13] copy done
 * [14] look-back rounds * 100000 + wait polls  [15] input slot free (pipelined kernel) */
#define DAQ_TRACE_WORDS 16

/*
 * Outputs (all device pointers, caller-owned).
 *   hdr, hdr_cap        island records, in (fill, calo, start) order.
 *   pool, pool_row_cap  pool rows, time-major: row r holds the n_xtal raw int16
 *                       samples of the r-th marked sample (row stride n_xtal
 *                       int16); 16-byte aligned.
 *   pedestal            int32[n_fills][n_calo][n_xtal] per-crystal pedestals, or NULL.
 *   counts              int64[4]: [0] islands found, [1] pool rows found (both
 *                       the full sizes, even when capacity ran out), [2] device
 *                       status bits DAQ_DEV_*, [3] tiles processed.  Readable
 *                       once the stream has reached the end of the call.
 * Records and rows beyond their capacity are not written (DAQ_DEV_*_OVERFLOW).
 */
typedef struct daq_islands {
    daq_island *hdr;
    int64_t hdr_cap;
    int16_t *pool;
    int64_t pool_row_cap;
    int32_t *pedestal;
    int64_t *counts;
} daq_islands;

/* Fill *p with the defaults: T = 30, pre = 8, post = 24, ped_samples = 100,
 * one decimation factor 32, everything else zero / NULL. */
void daq_params_default(daq_params *p);

/*
 * Bytes of device workspace daq_process_fills needs for these sizes and
 * parameters (tile choice, fills).  Returns DAQ_OK or DAQ_EINVAL.
 */
int daq_workspace_size(int n_calo, int n_xtal, int64_t n_samples, int n_fills, const daq_params *params,
                       size_t *bytes);

/*
 * Bins per calorimeter of the Q histogram for decimation factor D:
 * ceil(n_samples / D).  qhist_inout holds Q x bins(decim[0]) int64 values,
 * followed (if n_decim == 2) by Q x bins(decim[1]), Q = params->q_calos, or
 * n_calo when that is 0.
 */
int64_t daq_q_bins(int64_t n_samples, int32_t decim);

/*
 * Process n_fills fills of n_calo calorimeters in one launch sequence.
 *   samples      device int16[n_fills][n_calo][n_xtal][n_samples] (row pitch
 *                n_samples; 12-bit ADC values in 16-bit words, Sec. 3); the
 *                fast path wants 16-byte aligned rows (n_samples % 8 == 0).
 *   n_xtal       crystals per calorimeter, 1..64 (the experiment has 54, Sec. 3).
 *   qhist_inout  device int64 Q histograms (layout: see daq_q_bins); B_D[k] =
 *                sum of S over samples [kD, min(kD + D, len)) is ADDED to bin k
 *                of the fill's calorimeter for every fill (Table 2 rows 7-8).
 * Every output is an integer, so results are bit-exact and independent of
 * tile size, grid and scheduling.  Returns DAQ_OK once enqueued; with
 * DAQ_SYNC it waits and returns DAQ_ECAPACITY / DAQ_ETIMEOUT / DAQ_EINVAL
 * from counts[2].
 */
int daq_process_fills(const int16_t *samples, int n_calo, int n_xtal, int64_t n_samples, int n_fills,
                      const daq_params *params, const daq_islands *islands_out, int64_t *qhist_inout);

/*
 * Host buffers of daq_process_fills_host (the end-to-end form).
 *   samples_host   host int16[n_fills][n_calo][n_xtal][n_samples]; page-locked
 *                  memory gives full copy bandwidth.
 *   samples_dev    device buffer of the same size that receives the copy.
 *   hdr_host, pool_host, pedestal_host  host buffers that receive the island
 *                  records, pool rows and pedestals (pedestal_host may be NULL);
 *                  at most *_cap entries are copied.
 *   counts_host    host int64[4], receives counts (see daq_islands).
 *   With DAQ_PACK_POOL in params->flags the pool rows come back packed instead
 *   (pool_host is not used):
 *   packed_dev     device scratch for the packed streams, 16-byte aligned, of
 *                  at least daq_pack_bound(n_fills * n_calo * n_samples,
 *                  n_xtal) + 1024 bytes per chunk (64 chunks at most);
 *   packed_host    host buffer that receives one packed stream per chunk of
 *                  calorimeter-fills, back to back, in (fill, calo) order; each
 *                  stream decodes on its own (daq_unpack_pool) into that
 *                  chunk's pool rows, and the streams' rows concatenated are
 *                  the call's pool rows (the records' pool_row index them);
 *   packed_bytes_host  host int64, receives the total size of the streams.
 */
typedef struct daq_host_io {
    const int16_t *samples_host;
    int16_t *samples_dev;
    daq_island *hdr_host;
    int64_t hdr_host_cap;
    int16_t *pool_host;
    int64_t pool_host_cap;
    int32_t *pedestal_host;
    int64_t *counts_host;
    void *packed_dev;
    int64_t packed_dev_cap;
    uint8_t *packed_host;
    int64_t packed_host_cap;
    int64_t *packed_bytes_host;
} daq_host_io;

/*
 * End-to-end form over host buffers, as the paper's GPU thread does it (Sec. 3:
 * copy one fill to the GPU, process it, return the chopped islands to host
 * memory).  The call is cut into chunks of calorimeter-fills that are
 * pipelined: the copy of io->samples_host into io->samples_dev for one chunk
 * overlaps the processing of the previous chunk on params->stream and the
 * device-to-host copy of earlier chunks' island records and pool rows (exact
 * sizes).  On return, io->counts_host holds the call's counts and the host
 * buffers hold the records (in (fill, calo, start) order, pool_row indexing
 * pool_host), the pool rows and (if requested) the pedestals, exactly as
 * daq_process_fills would produce them.  The Q histograms stay on the device
 * (qhist_inout) and accumulate as with daq_process_fills.
 *   islands_dev  device buffers used as the chunks' working space: with
 *                capacity for every sample marked (pool_row_cap >= n_fills *
 *                n_calo * n_samples plus 8 rows per chunk, hdr_cap >= that
 *                many calorimeter-fills times ceil(n_samples / 2)) the call is
 *                pipelined, else it runs as one chunk.  Their contents after a
 *                pipelined call are per-chunk regions, not the call's layout;
 *                counts are reported in io->counts_host.
 *   params       as for daq_process_fills; params->workspace sized for the
 *                whole call.
 * Synchronous: returns when everything is on the host.  The first call on a
 * device creates two copy streams, events and a small page-locked count
 * buffer that live until the process exits; calls on one device are
 * serialised.  Returns the call's status (DAQ_ECAPACITY if a device or host
 * capacity was short: counts_host then holds the sizes needed).
 */
int daq_process_fills_host(int n_calo, int n_xtal, int64_t n_samples, int n_fills, const daq_params *params,
                           const daq_islands *islands_dev, int64_t *qhist_inout, const daq_host_io *io);

/*
 * Scratch-free variant (the paper has no counterpart: it concerns how this
 * library is called, not the method).  For callers that cannot allocate device
 * memory themselves - code living inside a memory budget fixed at start-up, a
 * plug-in whose host framework owns every device allocation, or a real-time
 * loop that must not call an allocator while taking data.  Arguments, outputs
 * and results are exactly those of daq_process_fills, except that the scratch
 * workspace comes from an area of DAQ_STATIC_SCRATCH_BYTES built into the
 * library (params->workspace and params->workspace_bytes are ignored).
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *   - The area exists once per GPU and lives until the process exits; every
 *     GPU that loads the library holds it.
 *   - The first call on a device looks up the area's device address (a
 *     runtime query, made once per device with that device current).  With
 *     the CUDA runtime's lazy module loading (the default) that first query is
 *     also when the area is placed in device memory, so inside a fixed memory
 *     budget make the first call at start-up, before the budget is spent; make
 *     it before any stream capture too.  Later calls place nothing.
 *   - The cached address belongs to the device's current context: after
 *     cudaDeviceReset the area is gone and this entry point must not be called
 *     again in that process.
 *   - Every call uses the same area, and it keeps what the last call left in
 *     it; each call re-initialises everything it reads.  Calls whose work
 *     overlaps on the GPU (different streams, or a second call enqueued before
 *     the first has run) race on the area and give wrong results: serialise
 *     them.
 *   - Returns DAQ_ESCRATCH, before touching the GPU, when the call needs more
 *     than DAQ_STATIC_SCRATCH_BYTES (daq_workspace_size() says how much); one
 *     full fill of 24 calorimeters x 54 crystals x 560,000 samples fits.
 */
#define DAQ_STATIC_SCRATCH_BYTES (8u << 20)
int daq_process_fills_static(const int16_t *samples, int n_calo, int n_xtal, int64_t n_samples, int n_fills,
                             const daq_params *params, const daq_islands *islands_out, int64_t *qhist_inout);

/*
 * Batch plans (the batching pattern: many calorimeter-fills of uneven length
 * and pulse rate in one launch).  A plan binds one batch - the same pointers,
 * sizes and parameters as daq_process_fills - to a tuned configuration and a
 * CUDA graph of the whole launch sequence, so that each daq_batch_launch is a
 * single graph launch with no host-side planning.
 *
 * daq_batch_plan_create
 *   samples ... qhist_inout  exactly as for daq_process_fills.  The graph reads
 *                the samples and params->fill_len (values may change between
 *                launches, pointers may not) and writes islands_out at every
 *                launch; qhist_inout receives each launch's bins.
 *   params       as for daq_process_fills; params->stream is not used (each
 *                launch names its stream).  params->workspace may be NULL: the
 *                plan then allocates and owns one.  With DAQ_TUNE, params->tile
 *                and params->grid are ignored and chosen by the tuner, and so
 *                is the DAQ_SPARSE bit of params->flags.
 *   plan_flags   DAQ_TUNE: time the candidate configurations (two-pass form at
 *                the library's tile, with and without DAQ_SPARSE, and at tile
 *                widths 128/224/384/448 with 2 or 1 CTAs per SM; the
 *                single-launch form at 448) on this batch and keep the
 *                fastest.  The choice is remembered per (device, sizes,
 *                windows, decimation, flags) for the rest of the process,
 *                whatever the data: a batch of the same shape whose islands
 *                are much sparser or denser (DAQ_SPARSE wins on one and not
 *                the other) should be tuned with DAQ_TUNE_FORCE.
 *                DAQ_TUNE_FORCE: ignore a remembered choice.
 *   *plan        receives the plan (NULL on error).
 * Creation is not the hot call: it may allocate, synchronises the device, and
 * runs the batch several times (tuning and a warm-up run) with islands_out as
 * output and a scratch Q histogram, so qhist_inout is untouched until the first
 * daq_batch_launch.  Returns DAQ_EINVAL for invalid arguments (checked before
 * any GPU work), else the status of the warm-up run or DAQ_ECUDA.
 *
 * daq_batch_launch       enqueue one replay on `stream` (cudaStream_t).  Replays
 *                        share the plan's workspace and outputs: serialise them.
 * daq_batch_plan_tuning  the chosen configuration and the timings behind it.
 * daq_batch_plan_destroy free the graph, stream and plan-owned workspace.
 * daq_tune_cache_clear   forget every remembered tuning choice.
 */
#define DAQ_TUNE 1u
#define DAQ_TUNE_FORCE 2u

typedef struct daq_batch_plan daq_batch_plan;

typedef struct daq_tune_result {
    int32_t tile;      /* chosen daq_params.tile */
    int32_t grid;      /* chosen daq_params.grid */
    int32_t n_tried;   /* candidates timed (0 if not tuned or taken from the cache) */
    int32_t from_cache;
    float ms;          /* mean time per run of the chosen candidate (ms), 0 if not timed */
    float ms_default;  /* the same for the default configuration (tile 0, grid 0) */
    uint32_t flags;    /* DAQ_SPARSE when the chosen configuration sets it, else 0 */
} daq_tune_result;

int daq_batch_plan_create(const int16_t *samples, int n_calo, int n_xtal, int64_t n_samples, int n_fills,
                          const daq_params *params, const daq_islands *islands_out, int64_t *qhist_inout,
                          uint32_t plan_flags, daq_batch_plan **plan);
int daq_batch_launch(daq_batch_plan *plan, void *stream);
int daq_batch_plan_tuning(const daq_batch_plan *plan, daq_tune_result *out);
int daq_batch_plan_destroy(daq_batch_plan *plan);
void daq_tune_cache_clear(void);

/*
 * Serving: a request loop that admits fills as they arrive (Sec. 3: fills
 * reach the GPU one after another during each accelerator cycle, and the Q
 * histograms are summed fill by fill).  A worker thread inside the server
 * admits every request whose arrival time has come as soon as a slot is free,
 * enqueues it on one of several streams, so that fills in flight overlap on
 * the device, and retires fills as their work completes.
 *
 *   slot   device memory for one fill: island records, pool rows, pedestals,
 *          counts, scratch workspace and (DAQ_SERVER_HOST_INPUT) an input
 *          buffer.  The server carves n_slots slots out of one allocation of
 *          at most mem_budget_bytes made at creation; a request waits in the
 *          queue while every slot is busy (admission against the budget).
 *   Q      one resident histogram (layout of daq_q_bins) that every fill adds
 *          to; the integer sums make the result independent of the order and
 *          overlap of fills.
 *   clock  microseconds since daq_server_create on the host's steady clock.
 *          Start and completion times come from CUDA events mapped onto that
 *          clock (re-anchored while the server is idle).
 *
 * daq_server_config fields:
 *   n_calo, n_xtal, n_samples  shape of every fill (row pitch n_samples).
 *   params          method parameters as for daq_process_fills (threshold,
 *                   windows, ped_samples, decimation, tile, grid); stream,
 *                   workspace, events, trace and fill_len are ignored.
 *   mem_budget_bytes  device bytes the slots may take (> 0).
 *   max_slots       upper bound on slots (0 = 64).
 *   n_streams       streams fills are spread over (0 = 4, at most 16).
 *   hdr_cap, pool_row_cap  per-fill output capacity (0 = worst case:
 *                   n_calo * n_samples rows, half that plus n_calo + 1 records).
 *   flags           DAQ_SERVER_HOST_INPUT: requests may name host samples,
 *                   copied into the slot's input buffer (page-locked memory
 *                   gives full speed) on one copy stream in admission order,
 *                   each fill's processing waiting for its own copy;
 *                   DAQ_SERVER_AUTO_RELEASE: a slot is freed
 *                   as soon as its fill completes (only counts and timings are
 *                   kept; for streaming without reading islands).
 *   qhist           device int64 Q histogram (caller-owned, accumulated), or
 *                   NULL for one owned by the server (zeroed at creation).
 */
#define DAQ_SERVER_HOST_INPUT 1u
#define DAQ_SERVER_AUTO_RELEASE 2u

typedef struct daq_server daq_server;

typedef struct daq_server_config {
    int32_t n_calo;
    int32_t n_xtal;
    int64_t n_samples;
    daq_params params;
    size_t mem_budget_bytes;
    int32_t max_slots;
    int32_t n_streams;
    int64_t hdr_cap;
    int64_t pool_row_cap;
    uint32_t flags;
    int32_t reserved;
    int64_t *qhist;
} daq_server_config;

/* Fill states */
#define DAQ_FILL_QUEUED 0
#define DAQ_FILL_RUNNING 1
#define DAQ_FILL_DONE 2
#define DAQ_FILL_RELEASED 3

/* Timing and size record of one fill (server clock, microseconds). */
typedef struct daq_fill_record {
    int64_t ticket;
    int64_t n_islands;
    int64_t n_rows;
    int64_t raw_bytes;   /* n_calo * n_xtal * fill_len * 2 */
    double t_arrival;    /* arrival (as submitted) */
    double t_admit;      /* slot granted and work enqueued (host) */
    double t_start;      /* work started on the GPU */
    double t_done;       /* work finished on the GPU */
    int32_t status;      /* daq_status of the fill */
    int32_t slot;
} daq_fill_record;

/* Result of one fill: its record plus device pointers into its slot (valid
 * until daq_server_release; NULL after AUTO_RELEASE). */
typedef struct daq_fill_result {
    daq_fill_record rec;
    int32_t state;
    int32_t reserved;
    const daq_island *hdr;
    const int16_t *pool;
    const int32_t *pedestal;
} daq_fill_result;

typedef struct daq_server_stats {
    int64_t submitted, admitted, completed, released, failed;
    int64_t queued, running, max_running;
    int32_t n_slots, n_streams;
    size_t slot_bytes, mem_bytes;
} daq_server_stats;

/* Latency / deadtime summary of completed fills (host arithmetic only). */
typedef struct daq_serving_summary {
    int64_t n;              /* fills summarised */
    double latency_p50_us;  /* t_done - t_arrival, percentiles with linear interpolation */
    double latency_p99_us;
    double latency_max_us;
    double deadtime;        /* over fills in arrival order that have a next fill: the fraction not
                               done before the next one arrives (0 when n < 2) */
    double gbs;             /* raw bytes / (last t_done - first t_arrival) / 1e3 (GB/s) */
    double span_us;
} daq_serving_summary;

/* Create the server: validates the configuration (DAQ_EINVAL before any GPU
 * work when invalid, or when the budget holds no slot), allocates the slots on
 * the current device and starts the worker thread. */
int daq_server_create(const daq_server_config *cfg, daq_server **out);
/* Queue one fill.  samples: device (or, with DAQ_SERVER_HOST_INPUT and
 * on_host != 0, host) int16[n_calo][n_xtal][n_samples]; it must stay valid and
 * unchanged until the fill completes.  fill_len in [0, n_samples] (-1 = n_samples).
 * arrival_us: server-clock arrival time; a future time holds the request until
 * then (replay), < 0 means now.  *ticket receives the fill's ticket (>= 1). */
int daq_server_submit(daq_server *s, const int16_t *samples, int on_host, int32_t fill_len, double arrival_us,
                      int64_t *ticket);
/* Non-blocking state of a ticket (DAQ_EINVAL for an unknown ticket). */
int daq_server_poll(daq_server *s, int64_t ticket, daq_fill_result *out);
/* Wait (up to timeout_s seconds) until the ticket is done; DAQ_ETIMEOUT otherwise. */
int daq_server_wait(daq_server *s, int64_t ticket, double timeout_s, daq_fill_result *out);
/* Copy a done (not yet released) fill's results to host buffers: up to
 * hdr_cap island records, pool_cap pool rows and (if ped_host != NULL)
 * n_calo x n_xtal pedestals.  Synchronous; DAQ_EINVAL unless the fill is done. */
int daq_server_fetch(daq_server *s, int64_t ticket, daq_island *hdr_host, int64_t hdr_cap, int16_t *pool_host,
                     int64_t pool_cap, int32_t *ped_host);
/* Free a done fill's slot. */
int daq_server_release(daq_server *s, int64_t ticket);
/* Wait (up to timeout_s) until nothing is queued or running. */
int daq_server_drain(daq_server *s, double timeout_s);
int daq_server_get_stats(daq_server *s, daq_server_stats *out);
/* Copy up to cap records of completed fills, in completion order; *n receives
 * how many exist.  clear != 0 forgets them afterwards. */
int daq_server_records(daq_server *s, daq_fill_record *out, int64_t cap, int64_t *n, int clear);
/* The resident Q histogram (device). */
int64_t *daq_server_qhist(daq_server *s);
/* Current server-clock time (microseconds). */
double daq_server_now_us(daq_server *s);
/* Stop the worker (after the work in flight completes) and free everything. */
int daq_server_destroy(daq_server *s);
/* Summarise records (any order): latency percentiles, deadtime, throughput. */
int daq_serving_summarize(const daq_fill_record *recs, int64_t n, daq_serving_summary *out);

/*
 * Per-crystal full-resolution fill sum (Table 2, fill-by-fill sum kernel in
 * the per-crystal, per-sample form its 30-million-thread count suggests).
 * For every fill f of the call, calorimeter c, crystal x and sample t < len_f:
 *     q_xtal[c][x][t] += samples[f][c][x][t] - P[f][c][x]
 * with P the crystal's pedestal as in daq_params.ped_samples (rounded half up).
 *   samples   device int16[n_fills][n_calo][n_xtal][n_samples].
 *   q_xtal    device int64[n_calo][n_xtal][n_samples], 16-byte aligned,
 *             accumulated (resident across calls); samples past a fill's
 *             length add nothing.
 *   params    ped_samples, fill_len (device, nullable; out-of-range lengths are
 *             clamped and flagged), stream, flags (DAQ_SYNC: wait and return
 *             DAQ_EINVAL if a fill length was out of range), workspace of at
 *             least daq_crystal_sum_workspace_size() bytes (16-byte aligned).
 *             Other fields are ignored.
 * Integer-exact; HBM traffic is the samples once plus q_xtal read and written
 * once per call (16 bytes per crystal-sample), so batching fills in one call
 * divides the Q traffic among them.
 */
int daq_crystal_sum_workspace_size(int n_calo, int n_xtal, int n_fills, size_t *bytes);
int daq_crystal_sum(const int16_t *samples, int n_calo, int n_xtal, int64_t n_samples, int n_fills,
                    const daq_params *params, int64_t *q_xtal);

/*
 * Lossless packing of pool rows (Sec. 3: the frontend compresses island data
 * losslessly before sending it to the event builder; the method is not named,
 * the format below is this library's).  Stream (little-endian):
 *   header   u32 magic 0x50514144, u32 n_xtal, u64 rows
 *   offsets  u64[n_blocks + 1], n_blocks = ceil(rows / 32): byte offset of each
 *            block's payload from the payload start (the last = payload size)
 *   payload  block b = rows [32b, 32b + 32), the last block padded with copies
 *            of its final row; per crystal x, with v_i the crystal's sample in
 *            row i of the block: z_0 = 0, z_i = zigzag(v_i - v_{i-1}) (2d for
 *            d >= 0, -2d - 1 otherwise), w = bit length of max z_i (0..17); the
 *            words (uint16)v_0 | w << 16, then w bit planes (bit i of plane k =
 *            bit k of z_i).
 * daq_pack_bound          worst-case stream bytes for rows x n_xtal (-1 if invalid).
 * daq_pack_workspace_size device scratch daq_pack_pool needs.
 * daq_pack_pool           pack device pool[rows][n_xtal] (n_xtal <= 64,
 *                         16-byte aligned) into device out (16-byte aligned,
 *                         out_cap bytes) on `stream`; *out_bytes (device
 *                         int64) receives the
 *                         stream's size - bytes past out_cap are not written,
 *                         so out_cap >= daq_pack_bound() is always enough -
 *                         or -1 when a copy of pool rows into shared memory
 *                         did not land within 4 s (the stream is then not
 *                         valid).
 * daq_unpack_pool         decode a stream of in_bytes bytes into device
 *                         pool_out[rows][n_xtal]; *err (device int32) is set
 *                         to 0, or to a non-zero code when the header does not
 *                         match (1) or the stream is malformed or cut short (2).
 * All asynchronous on `stream` (cudaStream_t); DAQ_EINVAL / DAQ_EUNSUPPORTED
 * for bad arguments before any device work.
 */
int64_t daq_pack_bound(int64_t rows, int n_xtal);
int daq_pack_workspace_size(int64_t rows, int n_xtal, size_t *bytes);
int daq_pack_pool(const int16_t *pool, int64_t rows, int n_xtal, void *out, int64_t out_cap, int64_t *out_bytes,
                  void *workspace, size_t workspace_bytes, void *stream);
int daq_unpack_pool(const void *in, int64_t in_bytes, int64_t rows, int n_xtal, int16_t *pool_out, int32_t *err,
                    void *stream);

/* Upper bound on the tiles of a call with these sizes and parameters (rows of
 * the trace buffer); 0 on invalid arguments. */
int64_t daq_trace_tiles(int n_calo, int n_xtal, int64_t n_samples, int n_fills, const daq_params *params);

/* Map a host copy of counts[4] to a daq_status (DAQ_OK if no bit is set). */
int daq_status_from_counts(const int64_t *counts_host);

/* Static, human-readable text for a daq_status. */
const char *daq_strerror(int status);

/* Name and text of the CUDA error behind the calling thread's last DAQ_ECUDA
 * from daq_process_fills (static storage; "no error" when there was none). */
const char *daq_last_cuda_error(void);

/* ABI version (major * 100 + minor). */
int daq_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DAQ_H */
