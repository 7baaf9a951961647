// Per-crystal full-resolution fill sum (Table 2, fill-by-fill sum kernel, in
// the form its thread count suggests: one term per crystal and sample):
//
//   Qx[c][x][t] += s[f][c][x][t] - P[f][c][x]   for every fill f and t < len_f
//
// with P the per-crystal pedestal of Table 2's pedestal kernel (the first
// min(ped_samples, len) samples, rounded half up).  Q stays on the device and
// accumulates over calls.  Two kernels: pedestals (one warp per crystal row),
// then a streaming pass in which each thread owns 8 consecutive samples of one
// crystal row, adds every fill of the call in registers and read-modify-writes
// its 8 int64 accumulators once.  HBM traffic per call: the samples once
// (2 bytes each) and Q once each way (16 bytes per crystal-sample).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "daq.h"

namespace daq_xtal {

constexpr int kThreads = 256;

struct XLayout {
    size_t status, lens, ped, total;
};

XLayout xlayout(int64_t n_fills, int64_t n_rows)
{
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    XLayout l;
    l.status = 0;
    l.lens = 256;
    l.ped = up(l.lens + sizeof(int32_t) * (size_t)std::max<int64_t>(n_fills, 1));
    l.total = up(l.ped + sizeof(int32_t) * (size_t)std::max<int64_t>(n_rows, 1));
    return l;
}

__device__ __forceinline__ long long floor_div_ll(long long a, long long b)
{
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// Fill lengths (clamped; out-of-range ones flagged in *status, cleared by the
// host before the launch) and every row's pedestal.
__global__ void __launch_bounds__(kThreads) xtal_prepare_kernel(const int16_t *samples, int n_fills, int n_calo,
                                                                int n_xtal, int64_t pitch, const int32_t *fill_len,
                                                                int ped_samples, int32_t *lens, int32_t *ped,
                                                                unsigned long long *status)
{
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * kThreads) >> 5;
    for (long long f = (long long)blockIdx.x * kThreads + threadIdx.x; f < n_fills; f += (long long)gridDim.x * kThreads) {
        long long len = fill_len ? (long long)fill_len[f] : pitch;
        if (len < 0 || len > pitch) {
            atomicOr(status, (unsigned long long)DAQ_DEV_BAD_FILL_LEN);
            len = len < 0 ? 0 : pitch;
        }
        lens[f] = (int32_t)len;
    }
    const long long n_rows = (long long)n_fills * n_calo * n_xtal;
    for (long long r = gw; r < n_rows; r += nw) {
        const long long f = r / ((long long)n_calo * n_xtal);
        long long len = fill_len ? (long long)fill_len[f] : pitch;
        len = len < 0 ? 0 : (len > pitch ? pitch : len);
        const long long n = len < ped_samples ? len : ped_samples;
        const int16_t *row = samples + r * pitch;
        long long sum = 0;
        for (long long t = lane; t < n; t += 32) sum += row[t];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
        if (lane == 0) ped[r] = n > 0 ? (int32_t)floor_div_ll(sum + n / 2, n) : 0;
    }
}

// kVec: rows 16-byte aligned (pitch % 8 == 0): 16-byte sample loads, 64-byte Q
// accesses; otherwise element by element.
template <bool kVec>
__global__ void __launch_bounds__(kThreads) xtal_sum_kernel(const int16_t *samples, int n_fills, int n_calo,
                                                            int n_xtal, int64_t pitch, const int32_t *lens,
                                                            const int32_t *ped, long long *q)
{
    const long long chunks = (pitch + 7) / 8;
    const long long n_rows = (long long)n_calo * n_xtal;
    const long long total = n_rows * chunks;
    const long long cx_stride = (long long)n_calo * n_xtal * pitch;  // one fill
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < total; i += (long long)gridDim.x * kThreads) {
        const long long row = i / chunks;
        const long long t0 = (i - row * chunks) * 8;
        long long acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0;
        long long *dst = q + row * pitch + t0;
        const bool vec_q = kVec && t0 + 8 <= pitch;
        longlong2 o[4];
        if (vec_q) {  // the accumulators' loads go out before the samples'
            const longlong2 *d2 = reinterpret_cast<const longlong2 *>(dst);
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = d2[k];
        }
        for (int f = 0; f < n_fills; ++f) {
            const long long len = lens[f];
            if (t0 >= len) continue;
            const int16_t *src = samples + (long long)f * cx_stride + row * pitch + t0;
            const long long P = ped[(long long)f * n_rows + row];
            if (kVec && t0 + 8 <= len) {
                const int4 v = __ldcs(reinterpret_cast<const int4 *>(src));  // streamed: read once
                const uint32_t w[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    acc[2 * k] += (long long)(int16_t)(w[k] & 0xffffu) - P;
                    acc[2 * k + 1] += (long long)(int16_t)(w[k] >> 16) - P;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (t0 + k < len) acc[k] += (long long)src[k] - P;
            }
        }
        if (vec_q) {
            longlong2 *d2 = reinterpret_cast<longlong2 *>(dst);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                o[k].x += acc[2 * k];
                o[k].y += acc[2 * k + 1];
                __stcs(d2 + k, o[k]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (t0 + k < pitch) dst[k] += acc[k];
        }
    }
}

int grid_for(long long work)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (work + kThreads - 1) / kThreads;
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)std::max(sms, 1) * 8));
}

}  // namespace daq_xtal

using namespace daq_xtal;

extern "C" {

int daq_crystal_sum_workspace_size(int n_calo, int n_xtal, int n_fills, size_t *bytes)
{
    if (!bytes || n_calo < 0 || n_xtal < 1 || n_fills < 0) return DAQ_EINVAL;
    *bytes = xlayout(n_fills, (int64_t)n_fills * n_calo * n_xtal).total;
    return DAQ_OK;
}

int daq_crystal_sum(const int16_t *samples, int n_calo, int n_xtal, int64_t n_samples, int n_fills,
                    const daq_params *params, int64_t *q_xtal)
{
    if (!params || n_calo < 0 || n_xtal < 1 || n_samples < 0 || n_fills < 0 || params->ped_samples < 1)
        return DAQ_EINVAL;
    const int64_t n_rows = (int64_t)n_fills * n_calo * n_xtal;
    const XLayout l = xlayout(n_fills, n_rows);
    if (!params->workspace || params->workspace_bytes < l.total ||
        (reinterpret_cast<uintptr_t>(params->workspace) & 15))
        return DAQ_EINVAL;
    const int64_t cells = (int64_t)n_calo * n_xtal * n_samples;
    if (cells > 0 && (!q_xtal || (reinterpret_cast<uintptr_t>(q_xtal) & 15))) return DAQ_EINVAL;
    if (n_rows * n_samples > 0 && !samples) return DAQ_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(params->stream);
    unsigned char *ws = static_cast<unsigned char *>(params->workspace);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(ws + l.status);
    int32_t *lens = reinterpret_cast<int32_t *>(ws + l.lens);
    int32_t *ped = reinterpret_cast<int32_t *>(ws + l.ped);
    if (cudaMemsetAsync(status, 0, sizeof(*status), s) != cudaSuccess) return DAQ_ECUDA;
    xtal_prepare_kernel<<<grid_for(std::max<int64_t>(n_rows * 32, n_fills)), kThreads, 0, s>>>(
        samples, n_fills, n_calo, n_xtal, n_samples, params->fill_len, params->ped_samples, lens, ped, status);
    if (cudaGetLastError() != cudaSuccess) return DAQ_ECUDA;
    if (cells > 0 && n_fills > 0) {
        const long long work = (long long)n_calo * n_xtal * ((n_samples + 7) / 8);
        const bool vec = n_samples % 8 == 0 && (reinterpret_cast<uintptr_t>(samples) & 15) == 0;
        if (vec)
            xtal_sum_kernel<true><<<grid_for(work), kThreads, 0, s>>>(samples, n_fills, n_calo, n_xtal, n_samples,
                                                                      lens, ped, reinterpret_cast<long long *>(q_xtal));
        else
            xtal_sum_kernel<false><<<grid_for(work), kThreads, 0, s>>>(samples, n_fills, n_calo, n_xtal, n_samples,
                                                                       lens, ped, reinterpret_cast<long long *>(q_xtal));
        if (cudaGetLastError() != cudaSuccess) return DAQ_ECUDA;
    }
    if (params->flags & DAQ_SYNC) {
        unsigned long long st = 0;
        if (cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return DAQ_ECUDA;
        if (st & DAQ_DEV_BAD_FILL_LEN) return DAQ_EINVAL;
    }
    return DAQ_OK;
}

}  // extern "C"
