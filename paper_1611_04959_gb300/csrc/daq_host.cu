// End-to-end form over host buffers (Sec. 3: the frontend's GPU thread copies
// one fill to the GPU, processes it and returns the chopped islands to host
// memory).  Copies are issued on the caller's stream around daq_process_fills.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "daq.h"

extern "C" int daq_process_fills_host(int n_calo, int n_xtal, int64_t n_samples, int n_fills,
                                      const daq_params *params, const daq_islands *dev, int64_t *qhist_inout,
                                      const daq_host_io *io)
{
    if (!params || !dev || !io || !io->counts_host || n_calo < 0 || n_xtal < 1 || n_samples < 0 || n_fills < 0)
        return DAQ_EINVAL;
    const size_t in_bytes = (size_t)n_fills * n_calo * n_xtal * n_samples * sizeof(int16_t);
    if (in_bytes && (!io->samples_host || !io->samples_dev)) return DAQ_EINVAL;
    const bool skip_isl = (params->flags & DAQ_SKIP_ISLANDS) != 0;
    if (!skip_isl && ((io->hdr_host_cap > 0 && !io->hdr_host) || (io->pool_host_cap > 0 && !io->pool_host) ||
                      io->hdr_host_cap < 0 || io->pool_host_cap < 0))
        return DAQ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(params->stream);

    if (in_bytes && cudaMemcpyAsync(io->samples_dev, io->samples_host, in_bytes, cudaMemcpyHostToDevice, s) !=
                        cudaSuccess)
        return DAQ_ECUDA;
    daq_params p = *params;
    p.flags &= ~DAQ_SYNC;
    int rc = daq_process_fills(io->samples_dev, n_calo, n_xtal, n_samples, n_fills, &p, dev, qhist_inout);
    if (rc != DAQ_OK) return rc;
    if (cudaMemcpyAsync(io->counts_host, dev->counts, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return DAQ_ECUDA;
    if (!skip_isl && io->pedestal_host && dev->pedestal) {
        const size_t pb = (size_t)n_fills * n_calo * n_xtal * sizeof(int32_t);
        if (pb && cudaMemcpyAsync(io->pedestal_host, dev->pedestal, pb, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return DAQ_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return DAQ_ECUDA;
    rc = daq_status_from_counts(io->counts_host);
    if (skip_isl) return rc;
    const int64_t n_isl = io->counts_host[0], n_rows = io->counts_host[1];
    const int64_t h = std::min(std::min(n_isl, dev->hdr_cap), io->hdr_host_cap);
    const int64_t r = std::min(std::min(n_rows, dev->pool_row_cap), io->pool_host_cap);
    if (h > 0 && cudaMemcpyAsync(io->hdr_host, dev->hdr, (size_t)h * sizeof(daq_island), cudaMemcpyDeviceToHost,
                                 s) != cudaSuccess)
        return DAQ_ECUDA;
    if (r > 0 && cudaMemcpyAsync(io->pool_host, dev->pool, (size_t)r * n_xtal * sizeof(int16_t),
                                 cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return DAQ_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DAQ_ECUDA;
    if (rc == DAQ_OK && (n_isl > io->hdr_host_cap || n_rows > io->pool_host_cap)) rc = DAQ_ECAPACITY;
    return rc;
}
