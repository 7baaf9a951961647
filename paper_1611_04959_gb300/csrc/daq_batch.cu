// Batch plans: one fixed batch of calorimeter-fills (uneven lengths allowed)
// processed by a tuned configuration and replayed as one CUDA graph launch.
//
// Plan creation (not the hot call) may allocate: the plan's workspace, a
// scratch Q histogram for the tuning and warm-up runs (so qhist_inout is only
// touched by daq_batch_launch), a private capture stream.  The autotuner runs
// each candidate configuration (form x tile width x CTAs per SM) on the
// caller's own batch, keeps the fastest, and remembers the choice per batch
// shape for the rest of the process.  Every candidate gives bit-identical
// results (all outputs are integers), so tuning only changes speed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "daq.h"

struct daq_batch_plan {
    int device = 0;
    const int16_t *samples = nullptr;
    int n_calo = 0, n_xtal = 0, n_fills = 0;
    int64_t n_samples = 0;
    daq_params p{};
    daq_islands isl{};
    int64_t *q = nullptr;
    void *own_ws = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    daq_tune_result tune{};
};

namespace {

using TuneKey = std::tuple<int, int, int, int64_t, int, int, int, int, int, int, int, int, uint32_t, int>;

std::mutex g_tune_mu;
std::map<TuneKey, std::tuple<int, int, uint32_t>> g_tune_cache;  // key -> (tile, grid, DAQ_SPARSE or 0)

TuneKey tune_key(int dev, int C, int X, int64_t N, int F, const daq_params &p)
{
    return TuneKey(dev, C, X, N, F, p.pre, p.post, p.ped_samples, p.n_decim, p.n_decim > 0 ? p.decim[0] : 0,
                   p.n_decim > 1 ? p.decim[1] : 0, p.fill_len != nullptr,
                   p.flags & (DAQ_SKIP_Q | DAQ_SKIP_ISLANDS), 0);
}

struct Candidate {
    int tile, grid;
    uint32_t flags;  // DAQ_SPARSE or 0
};

// Form x tile x CTAs: the default (two-pass, tile chosen by the library), the
// same with the compact pass that passes over tiles without marks (DAQ_SPARSE),
// the two-pass form at 128 / 224 / 384 / 448 with occupancy grids (2 CTAs per
// SM) and with one CTA per SM, and the single-launch form at 448.  The single-pass
// forms (plain, persistent, pipelined, streaming, single-read) are not timed:
// on every workload measured they were slower than the two-pass form.
std::vector<Candidate> candidates(int sms)
{
    return {{0, 0, 0u},   {0, 0, DAQ_SPARSE}, {448, 0, 0u},   {384, 0, 0u},
            {224, 0, 0u}, {128, 0, 0u},       {448, sms, 0u}, {224, sms, 0u}, {448, -4, 0u}};
}

int q_values(int64_t N, int C, const daq_params &p, int64_t *n)
{
    int64_t t = 0;
    for (int d = 0; d < p.n_decim && d < 2; ++d) {
        if (p.decim[d] < 1) return DAQ_EINVAL;
        t += (int64_t)C * daq_q_bins(N, p.decim[d]);
    }
    *n = t;
    return DAQ_OK;
}

// Grow `*ws` (plan-owned) to at least `need` bytes.
int ensure_ws(daq_batch_plan *pl, size_t need, size_t *have)
{
    if (need <= *have) return DAQ_OK;
    if (pl->own_ws) cudaFree(pl->own_ws);
    pl->own_ws = nullptr;
    *have = 0;
    if (cudaMalloc(&pl->own_ws, std::max<size_t>(need, 256)) != cudaSuccess) return DAQ_ECUDA;
    *have = need;
    return DAQ_OK;
}

// Run the batch once with configuration `c` on stream `s` (Q into `qs`).
int run_once(const daq_batch_plan *pl, const daq_params &base, Candidate c, void *ws, size_t ws_bytes, int64_t *qs,
             cudaStream_t s)
{
    daq_params p = base;
    p.tile = c.tile;
    p.grid = c.grid;
    p.flags = (p.flags & ~DAQ_SPARSE) | c.flags;
    p.stream = s;
    p.workspace = ws;
    p.workspace_bytes = ws_bytes;
    p.events = nullptr;
    p.trace = nullptr;
    p.flags &= ~DAQ_SYNC;
    return daq_process_fills(pl->samples, pl->n_calo, pl->n_xtal, pl->n_samples, pl->n_fills, &p, &pl->isl, qs);
}

void destroy(daq_batch_plan *pl)
{
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    if (pl->own_ws) cudaFree(pl->own_ws);
    delete pl;
}

}  // namespace

extern "C" {

int daq_batch_plan_create(const int16_t *samples, int n_calo, int n_xtal, int64_t n_samples, int n_fills,
                          const daq_params *params, const daq_islands *islands_out, int64_t *qhist_inout,
                          uint32_t plan_flags, daq_batch_plan **plan)
{
    if (!plan) return DAQ_EINVAL;
    *plan = nullptr;
    if (!params || !islands_out || n_calo < 0 || n_xtal < 1 || n_samples < 0 || n_fills < 0) return DAQ_EINVAL;
    if (plan_flags & ~(DAQ_TUNE | DAQ_TUNE_FORCE)) return DAQ_EINVAL;
    int64_t nq = 0;
    if (q_values(n_samples, n_calo, *params, &nq) != DAQ_OK) return DAQ_EINVAL;
    // Validate everything daq_process_fills checks on the host before any GPU work.
    size_t need0 = 0;
    int rc = daq_workspace_size(n_calo, n_xtal, n_samples, n_fills, params, &need0);
    if (rc != DAQ_OK) return rc;

    daq_batch_plan *pl = new daq_batch_plan();
    cudaGetDevice(&pl->device);
    pl->samples = samples;
    pl->n_calo = n_calo;
    pl->n_xtal = n_xtal;
    pl->n_samples = n_samples;
    pl->n_fills = n_fills;
    pl->p = *params;
    pl->p.flags &= ~DAQ_SYNC;
    pl->p.events = nullptr;
    pl->p.trace = nullptr;
    pl->isl = *islands_out;
    pl->q = qhist_inout;

    int64_t *qs = nullptr;  // scratch Q for tuning and warm-up
    auto fail = [&](int code) {
        if (qs) cudaFree(qs);
        destroy(pl);
        return code;
    };
    if (cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(DAQ_ECUDA);
    if (cudaMalloc(&qs, (size_t)std::max<int64_t>(nq, 1) * 8) != cudaSuccess) return fail(DAQ_ECUDA);

    // Caller workspace if given, else one owned by the plan (grown as candidates need).
    void *ws = params->workspace;
    size_t ws_bytes = params->workspace ? params->workspace_bytes : 0;
    const bool own = params->workspace == nullptr;
    size_t own_bytes = 0;

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
    Candidate best{params->tile, params->grid, params->flags & DAQ_SPARSE};
    pl->tune.tile = best.tile;
    pl->tune.grid = best.grid;
    const TuneKey key = tune_key(pl->device, n_calo, n_xtal, n_samples, n_fills, *params);
    bool cached = false;
    if ((plan_flags & DAQ_TUNE) && !(plan_flags & DAQ_TUNE_FORCE)) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = Candidate{std::get<0>(it->second), std::get<1>(it->second), std::get<2>(it->second)};
            cached = true;
        }
    }
    if ((plan_flags & DAQ_TUNE) && !cached) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            return fail(DAQ_ECUDA);
        }
        float best_ms = -1.f;
        int tried = 0;
        constexpr int kReps = 3;
        for (const Candidate &c : candidates(sms)) {
            daq_params pc = pl->p;
            pc.tile = c.tile;
            pc.grid = c.grid;
            pc.flags = (pc.flags & ~DAQ_SPARSE) | c.flags;
            size_t need = 0;
            if (daq_workspace_size(n_calo, n_xtal, n_samples, n_fills, &pc, &need) != DAQ_OK) continue;
            if (own) {
                if ((rc = ensure_ws(pl, need, &own_bytes)) != DAQ_OK) break;
                ws = pl->own_ws;
                ws_bytes = own_bytes;
            } else if (need > ws_bytes) {
                continue;  // the caller's workspace is too small for this candidate
            }
            if (run_once(pl, pl->p, c, ws, ws_bytes, qs, pl->cap) != DAQ_OK) continue;  // e.g. no fitting plan
            if (cudaStreamSynchronize(pl->cap) != cudaSuccess) {
                rc = DAQ_ECUDA;
                break;
            }
            cudaEventRecord(e0, pl->cap);
            for (int r = 0; r < kReps; ++r) run_once(pl, pl->p, c, ws, ws_bytes, qs, pl->cap);
            cudaEventRecord(e1, pl->cap);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = DAQ_ECUDA;
                break;
            }
            int64_t counts[4] = {0, 0, 0, 0};
            if (cudaMemcpy(counts, pl->isl.counts, sizeof(counts), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = DAQ_ECUDA;
                break;
            }
            if (counts[2] & (DAQ_DEV_TIMEOUT | DAQ_DEV_BAD_FILL_LEN)) continue;  // not a valid timing
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= kReps;
            ++tried;
            if (c.tile == 0 && c.grid == 0 && c.flags == 0u) pl->tune.ms_default = ms;
            if (best_ms < 0.f || ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != DAQ_OK) return fail(rc);
        if (tried == 0) return fail(DAQ_EINVAL);
        pl->tune.n_tried = tried;
        pl->tune.ms = best_ms;
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = std::make_tuple(best.tile, best.grid, best.flags);
    }
    pl->tune.tile = best.tile;
    pl->tune.grid = best.grid;
    pl->tune.flags = best.flags;
    pl->tune.from_cache = cached ? 1 : 0;
    pl->p.tile = best.tile;
    pl->p.grid = best.grid;
    pl->p.flags = (pl->p.flags & ~DAQ_SPARSE) | best.flags;

    size_t need = 0;
    if ((rc = daq_workspace_size(n_calo, n_xtal, n_samples, n_fills, &pl->p, &need)) != DAQ_OK) return fail(rc);
    if (own) {
        if ((rc = ensure_ws(pl, need, &own_bytes)) != DAQ_OK) return fail(rc);
        ws = pl->own_ws;
        ws_bytes = own_bytes;
    } else if (need > ws_bytes) {
        return fail(DAQ_EINVAL);
    }
    pl->p.workspace = ws;
    pl->p.workspace_bytes = ws_bytes;

    // Warm-up outside capture (sets per-kernel attributes once), then capture.
    if ((rc = run_once(pl, pl->p, best, ws, ws_bytes, qs, pl->cap)) != DAQ_OK) return fail(rc);
    if (cudaStreamSynchronize(pl->cap) != cudaSuccess) return fail(DAQ_ECUDA);
    cudaFree(qs);
    qs = nullptr;
    daq_params pcap = pl->p;
    pcap.stream = pl->cap;
    if (cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(DAQ_ECUDA);
    rc = daq_process_fills(samples, n_calo, n_xtal, n_samples, n_fills, &pcap, &pl->isl, qhist_inout);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(pl->cap, &g);
    pl->graph = g;
    if (rc != DAQ_OK) return fail(rc);
    if (ce != cudaSuccess || !g) return fail(DAQ_ECUDA);
    if (cudaGraphInstantiate(&pl->exec, g, 0) != cudaSuccess) return fail(DAQ_ECUDA);
    *plan = pl;
    return DAQ_OK;
}

int daq_batch_launch(daq_batch_plan *plan, void *stream)
{
    if (!plan || !plan->exec) return DAQ_EINVAL;
    return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? DAQ_OK : DAQ_ECUDA;
}

int daq_batch_plan_tuning(const daq_batch_plan *plan, daq_tune_result *out)
{
    if (!plan || !out) return DAQ_EINVAL;
    *out = plan->tune;
    return DAQ_OK;
}

int daq_batch_plan_destroy(daq_batch_plan *plan)
{
    if (!plan) return DAQ_EINVAL;
    destroy(plan);
    return DAQ_OK;
}

void daq_tune_cache_clear(void)
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache.clear();
}

}  // extern "C"
