// daq_process_fills_static: the same processing as daq_process_fills, for
// callers that cannot allocate device memory themselves (for example code that
// runs inside a fixed memory budget carved out at start-up, a plug-in whose
// host framework owns every device allocation, or a real-time loop that must
// not call an allocator once data taking has started).  Such a caller still
// passes its input and output buffers; only the scratch workspace comes from a
// fixed-size area built into this library.
//
// The area is a file-scope __device__ array, so every GPU that loads the
// library holds DAQ_STATIC_SCRATCH_BYTES of it until the process exits.  Host
// code cannot hand the array's name to a kernel (on the host that name is only
// a stand-in, not a device address), so the first call on each device asks the
// runtime for the array's device address once, with that device current, and
// keeps it.  Under lazy module loading that first query is also when the
// module, and with it the area, is placed on the device; the address is that
// of the current context and does not survive cudaDeviceReset.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "daq.h"

static __device__ __align__(256) unsigned char g_daq_static_scratch[DAQ_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch area on the current device (set up on first use).
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DAQ_ECUDA;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_daq_static_scratch) != cudaSuccess || !p) return DAQ_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return DAQ_OK;
}

}  // namespace

extern "C" int daq_process_fills_static(const int16_t *samples, int n_calo, int n_xtal, int64_t n_samples,
                                        int n_fills, const daq_params *params, const daq_islands *islands_out,
                                        int64_t *qhist_inout)
{
    if (!params) return DAQ_EINVAL;
    size_t need = 0;
    int rc = daq_workspace_size(n_calo, n_xtal, n_samples, n_fills, params, &need);
    if (rc != DAQ_OK) return rc;
    if (need > (size_t)DAQ_STATIC_SCRATCH_BYTES) return DAQ_ESCRATCH;
    void *scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != DAQ_OK) return rc;
    // The processing resets every scratch field it reads before writing it
    // (tile plan, counters, scan state), so nothing is cleared here.
    daq_params p;
    std::memcpy(&p, params, sizeof(p));
    p.workspace = scratch;
    p.workspace_bytes = DAQ_STATIC_SCRATCH_BYTES;
    return daq_process_fills(samples, n_calo, n_xtal, n_samples, n_fills, &p, islands_out, qhist_inout);
}
