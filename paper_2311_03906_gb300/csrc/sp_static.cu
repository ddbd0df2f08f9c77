// sp_static.cu -- sp_sample_static: sampling that allocates no memory.
//
// Some callers cannot call cudaMalloc: a process whose GPU memory is already
// reserved in full by another allocator (a caching allocator or a memory
// pool that owns the device), code on a latency-critical path where an
// allocation's implicit device synchronisation is not acceptable, or a host
// application whose plugin rules forbid extensions from allocating device
// memory.  sp_sample allocates its fault-bit and record tiles the first time
// it needs them; this entry point instead works in one fixed array that the
// library reserves when its code is loaded on a device.
#include <algorithm>
#include <mutex>
#include <string>

#include "sp_internal.h"

namespace sp {

// The fixed scratch: fault bits and bit-sliced records of one chunk of shots.
// Every GPU that loads the library holds it until the process exits.
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) uint32_t g_static_scratch[STATIC_SCRATCH_BYTES / sizeof(uint32_t)];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
uint32_t *g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the array on device dev, which must be current.  The
// host-side symbol g_static_scratch is only a stand-in for it and must never
// be passed to a kernel, so the address is looked up once per device, with
// that device current, and cached for the life of the process (the cache
// assumes the device's primary context is not reset meanwhile).
sp_status scratch_for_device(int dev, uint32_t **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(SP_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return set_error(SP_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                              cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = static_cast<uint32_t *>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return SP_OK;
}
}  // namespace

}  // namespace sp

using namespace sp;

extern "C" sp_status sp_sample_static(sp_program *P, uint64_t seed, uint64_t shot0, uint64_t nshots,
                                      uint64_t *d_meas, uint64_t *d_det, uint64_t *d_obs,
                                      void *cuda_stream)
{
    if (!P) return set_error(SP_ERR_INVALID_ARG, "prog is NULL");
    for (const void *p : {(const void *)d_meas, (const void *)d_det, (const void *)d_obs})
        if (p && (reinterpret_cast<uintptr_t>(p) & 7u))
            return set_error(SP_ERR_INVALID_ARG, "output pointer is not 8-byte aligned");
    if (shot0 + nshots < shot0) return set_error(SP_ERR_INVALID_ARG, "shot range overflows 64 bits");
    // One 32-shot word of every fault-symbol row and every record row must fit.
    const uint64_t rows = (uint64_t)std::max<int64_t>(P->n_sym, 0) + (uint64_t)std::max<int64_t>(P->n_rows, 0);
    const uint64_t words_total = STATIC_SCRATCH_BYTES / sizeof(uint32_t);
    const uint64_t pitch = rows ? words_total / rows : words_total;
    if (pitch == 0)
        return set_error(SP_ERR_TOO_LARGE,
                         "program needs " + std::to_string(rows * 4) + " bytes per 32 shots; the static scratch holds " +
                             std::to_string(STATIC_SCRATCH_BYTES) + " bytes");
    if (P->stream != 1)
        return set_error(SP_ERR_INVALID_ARG, "the static-scratch entry point draws the per-channel stream (stream 1) only");
    if (nshots == 0) return SP_OK;
    // the program's tables and the scratch must live on the same GPU
    int dev = -1;
    SP_CUDA(cudaGetDevice(&dev));
    if (dev != P->device)
        return set_error(SP_ERR_INVALID_ARG, "the program lives on device " + std::to_string(P->device) +
                                                 " but device " + std::to_string(dev) + " is current");
    uint32_t *base = nullptr;
    sp_status st = scratch_for_device(dev, &base);
    if (st != SP_OK) return st;
    uint32_t *B = base;
    uint32_t *recT = base + (size_t)std::max<int64_t>(P->n_sym, 0) * pitch;
    const uint64_t chunk = pitch * 32;
    const int64_t wm = (P->n_meas + 63) / 64, wd = (P->n_det + 63) / 64, wo = (P->n_obs + 63) / 64;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // Every row of every word that a chunk reads is written earlier in the
    // same chunk, so nothing in the array has to start at zero.
    for (uint64_t done = 0; done < nshots;) {
        const uint64_t n = std::min<uint64_t>(nshots - done, chunk);
        st = sample_chunk_into(P, B, recT, (int64_t)pitch, seed, shot0 + done, n,
                               d_meas ? d_meas + done * wm : nullptr, d_det ? d_det + done * wd : nullptr,
                               d_obs ? d_obs + done * wo : nullptr, s);
        if (st != SP_OK) return st;
        done += n;
    }
    return SP_OK;
}
