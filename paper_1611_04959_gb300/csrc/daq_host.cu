// End-to-end form over host buffers (Sec. 3: the frontend's GPU thread copies
// one fill to the GPU, processes it and returns the chopped islands to host
// memory).
//
// The call is cut into chunks of calorimeter-fills (a group of calorimeters of
// one fill, or whole fills) and pipelined over three streams: the host->device
// copy of chunk j+1 runs while chunk j is processed on the caller's stream,
// and chunk j's island records and pool rows travel back on a third stream,
// with their exact sizes, while later chunks are copied in and processed.
// Each chunk writes its outputs to its own region of the device buffers; the
// host copies land back to back, and the pool rows of a chunk's records are
// shifted by the rows of the chunks before it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include "daq.h"

namespace {

constexpr int kMaxChunks = 64;
constexpr int kTargetChunks = 12;        // rows copied back as they are
constexpr int kTargetChunksPacked = 24;  // rows packed on the GPU first
// make_chunks may return up to about twice its target (whole fills, or groups
// of calorimeters, rounded), and every per-chunk array holds kMaxChunks
static_assert(2 * kTargetChunks <= kMaxChunks && 2 * kTargetChunksPacked <= kMaxChunks,
              "chunk plans must fit the per-chunk arrays");
constexpr int kMaxDevices = 64;

// Streams, events and count buffers of the pipeline, created on a device's
// first call and kept for the life of the process.
struct HostPipe {
    std::mutex call;  // one call at a time per device
    bool ready = false;
    cudaStream_t h2d = nullptr, d2h = nullptr, pk = nullptr;
    cudaEvent_t entry = nullptr;
    cudaEvent_t in_ev[kMaxChunks] = {}, proc_ev[kMaxChunks] = {}, pack_ev[kMaxChunks] = {};
    int64_t *counts_d = nullptr;  // [kMaxChunks][4] device
    int64_t *counts_h = nullptr;  // [kMaxChunks][4] page-locked
    int64_t *psize_d = nullptr;   // [kMaxChunks] packed stream sizes, device
    int64_t *psize_h = nullptr;   // [kMaxChunks] page-locked
    void *pack_ws = nullptr;      // packing scratch, grown on demand
    size_t pack_ws_bytes = 0;
};

std::mutex g_mu;
HostPipe g_pipe[kMaxDevices];

int pipe_for(int dev, HostPipe **out)
{
    if (dev < 0 || dev >= kMaxDevices) return DAQ_ECUDA;
    std::lock_guard<std::mutex> g(g_mu);
    HostPipe &hp = g_pipe[dev];
    if (!hp.ready) {
        if (cudaStreamCreateWithFlags(&hp.h2d, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&hp.d2h, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&hp.pk, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&hp.entry, cudaEventDisableTiming) != cudaSuccess)
            return DAQ_ECUDA;
        for (int j = 0; j < kMaxChunks; ++j)
            if (cudaEventCreateWithFlags(&hp.in_ev[j], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&hp.proc_ev[j], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&hp.pack_ev[j], cudaEventDisableTiming) != cudaSuccess)
                return DAQ_ECUDA;
        if (cudaMalloc(&hp.counts_d, sizeof(int64_t) * 4 * kMaxChunks) != cudaSuccess ||
            cudaMallocHost(&hp.counts_h, sizeof(int64_t) * 4 * kMaxChunks) != cudaSuccess ||
            cudaMalloc(&hp.psize_d, sizeof(int64_t) * kMaxChunks) != cudaSuccess ||
            cudaMallocHost(&hp.psize_h, sizeof(int64_t) * kMaxChunks) != cudaSuccess)
            return DAQ_ECUDA;
        hp.ready = true;
    }
    *out = &hp;
    return DAQ_OK;
}

struct Chunk {
    int f0, nf, c0, nc;
    int64_t hdr_off, hdr_cap, row_off, row_cap;  // device regions (records, rows)
    int64_t isl_at, isl_copied, rows_before;     // host placement
    int64_t pk_off, pk_cap;                      // device region of the packed stream
};

// Chunks of about U / target calorimeter-fills, never splitting a
// calorimeter-fill and never mixing parts of two fills.
std::vector<Chunk> make_chunks(int F, int C, int target)
{
    std::vector<Chunk> v;
    const int64_t U = (int64_t)F * C;
    if (U == 0) return v;
    const int64_t u = (U + target - 1) / target;
    if (u >= C) {
        const int m = (int)(u / C);
        for (int f = 0; f < F; f += m) v.push_back(Chunk{f, std::min(m, F - f), 0, C, 0, 0, 0, 0, 0, 0, 0, 0, 0});
    } else {
        for (int f = 0; f < F; ++f)
            for (int c = 0; c < C; c += (int)u) v.push_back(Chunk{f, 1, c, std::min((int)u, C - c), 0, 0, 0, 0, 0, 0, 0, 0, 0});
    }
    return v;
}

}  // namespace

extern "C" int daq_process_fills_host(int n_calo, int n_xtal, int64_t n_samples, int n_fills,
                                      const daq_params *params, const daq_islands *dev, int64_t *qhist_inout,
                                      const daq_host_io *io)
{
    if (!params || !dev || !io || !io->counts_host || n_calo < 0 || n_xtal < 1 || n_samples < 0 || n_fills < 0)
        return DAQ_EINVAL;
    const int64_t C = n_calo, X = n_xtal, N = n_samples;
    const size_t cf_bytes = (size_t)(X * N) * sizeof(int16_t);
    const size_t in_bytes = (size_t)n_fills * C * cf_bytes;
    if (in_bytes && (!io->samples_host || !io->samples_dev)) return DAQ_EINVAL;
    const bool skip_isl = (params->flags & DAQ_SKIP_ISLANDS) != 0;
    if (!skip_isl && ((io->hdr_host_cap > 0 && !io->hdr_host) || (io->pool_host_cap > 0 && !io->pool_host) ||
                      io->hdr_host_cap < 0 || io->pool_host_cap < 0))
        return DAQ_EINVAL;
    if (!dev->counts) return DAQ_EINVAL;
    const bool pack = (params->flags & DAQ_PACK_POOL) != 0 && !skip_isl;
    if (pack && (!io->packed_dev || io->packed_dev_cap < 0 || (reinterpret_cast<uintptr_t>(io->packed_dev) & 15) ||
                 !io->packed_bytes_host || io->packed_host_cap < 0 || (io->packed_host_cap > 0 && !io->packed_host)))
        return DAQ_EINVAL;
    // Validate the whole call (sizes, parameters, workspace) before any copy.
    size_t need = 0;
    int rc = daq_workspace_size(n_calo, n_xtal, n_samples, n_fills, params, &need);
    if (rc != DAQ_OK) return rc;
    if (!params->workspace || params->workspace_bytes < need) return DAQ_EINVAL;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return DAQ_ECUDA;
    HostPipe *hp = nullptr;
    if ((rc = pipe_for(device, &hp)) != DAQ_OK) return rc;
    std::lock_guard<std::mutex> call_lock(hp->call);
    cudaStream_t s = static_cast<cudaStream_t>(params->stream);

    // Chunk plan; each chunk's device region holds its worst case (every
    // sample marked; an island per two samples), rows rounded to 8 so every
    // region starts 16-byte aligned.  Too little device capacity: one chunk.
    std::vector<Chunk> ch = make_chunks(n_fills, n_calo, pack ? kTargetChunksPacked : kTargetChunks);
    if (ch.empty()) ch.push_back(Chunk{0, n_fills, 0, n_calo, 0, 0, 0, 0, 0, 0, 0, 0, 0});
    {
        int64_t h = 0, r = 0;
        for (Chunk &c : ch) {
            const int64_t units = (int64_t)c.nf * c.nc;
            c.hdr_off = h;
            c.hdr_cap = units * ((N + 1) / 2);
            c.row_off = r;
            c.row_cap = units * N;
            h += c.hdr_cap;
            r += (c.row_cap + 7) & ~int64_t(7);
        }
        if (ch.size() > 1 && !skip_isl && (h > dev->hdr_cap || r > dev->pool_row_cap)) ch.resize(1);
        if (ch.size() > (size_t)kMaxChunks) ch.resize(1);  // more chunks than the per-chunk arrays hold: one chunk
        if (ch.size() == 1) {
            ch[0] = Chunk{0, n_fills, 0, n_calo, 0, dev->hdr_cap, 0, dev->pool_row_cap, 0, 0, 0, 0, 0};
        }
    }
    const int nch = (int)ch.size();
    if (pack) {
        int64_t off = 0;
        size_t ws_need = 0;
        for (Chunk &c : ch) {
            c.pk_off = off;
            c.pk_cap = (daq_pack_bound(c.row_cap, n_xtal) + 15) & ~int64_t(15);
            off += c.pk_cap;
            size_t w = 0;
            if (daq_pack_workspace_size(c.row_cap, n_xtal, &w) != DAQ_OK) return DAQ_EINVAL;
            ws_need = std::max(ws_need, w);
        }
        if (off > io->packed_dev_cap) return DAQ_EINVAL;
        if (ws_need > hp->pack_ws_bytes) {  // grown once per device and size
            if (hp->pack_ws) cudaFree(hp->pack_ws);
            hp->pack_ws = nullptr;
            hp->pack_ws_bytes = 0;
            if (cudaMalloc(&hp->pack_ws, ws_need) != cudaSuccess) return DAQ_ECUDA;
            hp->pack_ws_bytes = ws_need;
        }
    }

    // Enqueue every copy-in and every chunk's processing up front.
    if (cudaEventRecord(hp->entry, s) != cudaSuccess || cudaStreamWaitEvent(hp->h2d, hp->entry, 0) != cudaSuccess)
        return DAQ_ECUDA;
    int enq = 0;
    for (int j = 0; j < nch && rc == DAQ_OK; ++j) {
        const Chunk &c = ch[j];
        const size_t off = ((size_t)c.f0 * C + c.c0) * cf_bytes;
        const size_t bytes = (size_t)c.nf * c.nc * cf_bytes;
        const int16_t *src = reinterpret_cast<const int16_t *>(reinterpret_cast<const unsigned char *>(io->samples_host) + off);
        int16_t *dst = reinterpret_cast<int16_t *>(reinterpret_cast<unsigned char *>(io->samples_dev) + off);
        if (bytes && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, hp->h2d) != cudaSuccess) {
            rc = DAQ_ECUDA;
            break;
        }
        if (cudaEventRecord(hp->in_ev[j], hp->h2d) != cudaSuccess || cudaStreamWaitEvent(s, hp->in_ev[j], 0) != cudaSuccess) {
            rc = DAQ_ECUDA;
            break;
        }
        daq_params p = *params;
        p.flags &= ~(DAQ_SYNC | DAQ_PACK_POOL);
        p.events = nullptr;
        p.trace = nullptr;
        p.fill_base = params->fill_base + c.f0;
        p.fill_len = params->fill_len ? params->fill_len + c.f0 : nullptr;
        p.calo_base = params->calo_base + c.c0;
        p.q_calos = params->q_calos > 0 ? params->q_calos : n_calo;
        daq_islands isl;
        isl.hdr = dev->hdr ? dev->hdr + c.hdr_off : nullptr;
        isl.hdr_cap = c.hdr_cap;
        isl.pool = dev->pool ? dev->pool + c.row_off * X : nullptr;
        isl.pool_row_cap = c.row_cap;
        isl.pedestal = dev->pedestal ? dev->pedestal + ((int64_t)c.f0 * C + c.c0) * X : nullptr;
        isl.counts = nch == 1 ? dev->counts : hp->counts_d + 4 * j;
        rc = daq_process_fills(dst, c.nc, n_xtal, n_samples, c.nf, &p, &isl, qhist_inout);
        if (rc != DAQ_OK) break;
        if (cudaMemcpyAsync(hp->counts_h + 4 * j, isl.counts, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaEventRecord(hp->proc_ev[j], s) != cudaSuccess) {
            rc = DAQ_ECUDA;
            break;
        }
        ++enq;
    }

    // Copy each chunk's results back as soon as it is done.  Packed form: the
    // chunk's pool is packed on its own stream right away, and its stream
    // (size read back with it) travels once the next chunk has been handed over.
    int64_t tot_isl = 0, tot_rows = 0, tot_tiles = 0, bits = 0, packed_at = 0;
    int pending = -1;  // chunk whose packed stream is still to be copied back
    auto finish_pack = [&](int j) {
        if (cudaEventSynchronize(hp->pack_ev[j]) != cudaSuccess) {
            rc = DAQ_ECUDA;
            return;
        }
        const int64_t n = hp->psize_h[j];
        if (n < 0) {  // the packing gave up (a block copy did not land)
            rc = DAQ_ETIMEOUT;
            return;
        }
        const int64_t k = std::max<int64_t>(0, std::min(n, io->packed_host_cap - packed_at));
        if (k > 0 && cudaMemcpyAsync(io->packed_host + packed_at, static_cast<unsigned char *>(io->packed_dev) + ch[j].pk_off,
                                     (size_t)k, cudaMemcpyDeviceToHost, hp->d2h) != cudaSuccess)
            rc = DAQ_ECUDA;
        packed_at += n;
    };
    for (int j = 0; j < enq; ++j) {
        if (cudaEventSynchronize(hp->proc_ev[j]) != cudaSuccess) {
            rc = DAQ_ECUDA;
            break;
        }
        if (rc != DAQ_OK) continue;  // a later chunk failed to enqueue: only wait
        const int64_t *cnt = hp->counts_h + 4 * j;
        Chunk &c = ch[j];
        c.isl_at = tot_isl;
        c.rows_before = tot_rows;
        bits |= cnt[2];
        tot_tiles += cnt[3];
        if (!skip_isl) {
            const int64_t h = std::max<int64_t>(0, std::min(std::min(cnt[0], c.hdr_cap), io->hdr_host_cap - tot_isl));
            const int64_t r = std::max<int64_t>(0, std::min(std::min(cnt[1], c.row_cap), io->pool_host_cap - tot_rows));
            c.isl_copied = h;
            if (h > 0 && cudaMemcpyAsync(io->hdr_host + tot_isl, dev->hdr + c.hdr_off, (size_t)h * sizeof(daq_island),
                                         cudaMemcpyDeviceToHost, hp->d2h) != cudaSuccess)
                rc = DAQ_ECUDA;
            if (pack) {
                const int64_t rows_j = std::min(cnt[1], c.row_cap);
                if (cudaStreamWaitEvent(hp->pk, hp->proc_ev[j], 0) != cudaSuccess ||
                    daq_pack_pool(dev->pool + c.row_off * X, rows_j, n_xtal,
                                  static_cast<unsigned char *>(io->packed_dev) + c.pk_off, c.pk_cap, hp->psize_d + j,
                                  hp->pack_ws, hp->pack_ws_bytes, hp->pk) != DAQ_OK ||
                    cudaMemcpyAsync(hp->psize_h + j, hp->psize_d + j, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    hp->pk) != cudaSuccess ||
                    cudaEventRecord(hp->pack_ev[j], hp->pk) != cudaSuccess)
                    rc = DAQ_ECUDA;
                if (rc == DAQ_OK && pending >= 0) finish_pack(pending);
                pending = j;
            } else if (r > 0 && cudaMemcpyAsync(io->pool_host + tot_rows * X, dev->pool + c.row_off * X,
                                                (size_t)(r * X) * sizeof(int16_t), cudaMemcpyDeviceToHost, hp->d2h) !=
                                    cudaSuccess) {
                rc = DAQ_ECUDA;
            }
        }
        tot_isl += cnt[0];
        tot_rows += cnt[1];
    }
    if (rc == DAQ_OK && pending >= 0) finish_pack(pending);
    if (enq < nch || rc != DAQ_OK) {  // something failed: let the work in flight finish
        cudaStreamSynchronize(hp->h2d);
        cudaStreamSynchronize(s);
        cudaStreamSynchronize(hp->pk);
    }
    if (rc == DAQ_OK && !skip_isl && io->pedestal_host && dev->pedestal) {
        const size_t pb = (size_t)n_fills * C * X * sizeof(int32_t);
        if (pb && cudaMemcpyAsync(io->pedestal_host, dev->pedestal, pb, cudaMemcpyDeviceToHost, hp->d2h) != cudaSuccess)
            rc = DAQ_ECUDA;
    }
    if (cudaStreamSynchronize(hp->d2h) != cudaSuccess && rc == DAQ_OK) rc = DAQ_ECUDA;
    if (rc != DAQ_OK) return rc;

    // Pool rows of each chunk's records: shift by the rows of earlier chunks.
    if (!skip_isl && nch > 1)
        for (const Chunk &c : ch)
            for (int64_t i = 0; i < c.isl_copied; ++i) io->hdr_host[c.isl_at + i].pool_row += c.rows_before;
    if (pack) *io->packed_bytes_host = packed_at;
    io->counts_host[0] = tot_isl;
    io->counts_host[1] = tot_rows;
    io->counts_host[2] = bits;
    io->counts_host[3] = tot_tiles;
    rc = daq_status_from_counts(io->counts_host);
    if (rc == DAQ_OK && !skip_isl &&
        (tot_isl > io->hdr_host_cap || (pack ? packed_at > io->packed_host_cap : tot_rows > io->pool_host_cap)))
        rc = DAQ_ECAPACITY;
    return rc;
}
