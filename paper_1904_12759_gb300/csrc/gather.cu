// Random-gather ceiling: the rate at which this GPU serves loads of random
// 32-byte sectors from a buffer that fits in L2 and from one far larger than
// L2.  It is the measured roofline of the walkers, whose every jump is two such
// gathers (a column and a node record).
//
// Each thread performs `steps` loads of 16 bytes, each from a random sector of
// the buffer (the sector is fetched whole).  Independent mode: the sector
// indices come from a counter hash, so a thread's loads can all be in flight.
// Dependent mode: the next index hashes the loaded word, so each thread is a
// chain of dependent loads, as a walker is.  Indices map a 32-bit hash to
// [0, sectors) by a multiply-high (sectors < 2^32).  The hash is the 32-bit
// finaliser of MurmurHash3 (Appleby).
#include <stdint.h>

#include "launch.h"
#include "mcx_internal.cuh"

namespace mcx {
namespace {

constexpr int GATHER_THREADS = 256;
constexpr int GATHER_BLOCKS_PER_SM = 8;

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__global__ void __launch_bounds__(GATHER_THREADS) k_gather(const int4 *__restrict__ buf, uint32_t sectors,
                                                           uint32_t steps, int dependent, uint32_t seed,
                                                           uint32_t *__restrict__ sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x = fmix32(tid ^ seed);
    uint32_t acc = 0;
    for (uint32_t k = 0; k < steps; ++k) {
        const uint32_t idx = __umulhi(x, sectors);  // < sectors
        const int4 w = __ldg(buf + 2ull * idx);     // first 16 bytes of the 32-byte sector
        acc ^= (uint32_t)w.x;
        x = dependent ? fmix32((uint32_t)w.x ^ x ^ k) : fmix32(x + 0x9E3779B9u);
    }
    sink[tid & 1023u] = acc;  // keeps the loads; the sink's contents are never read
}

}  // namespace
}  // namespace mcx

extern "C" {

mcx_status mcx_gather_rate(uint64_t buffer_bytes, int dependent, uint64_t loads, double *sectors_per_second,
                           void *stream) {
    if (!sectors_per_second || buffer_bytes < (1ull << 20) || buffer_bytes > (1ull << 37) || loads < 1)
        return MCX_E_INVALID;
    const uint64_t sectors64 = buffer_bytes / 32;
    if (sectors64 >= (1ull << 32)) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return MCX_E_CUDA;
    const unsigned grid = (unsigned)sms * mcx::GATHER_BLOCKS_PER_SM;
    const uint64_t threads = (uint64_t)grid * mcx::GATHER_THREADS;
    const uint64_t steps64 = (loads + threads - 1) / threads;
    if (steps64 > 0xFFFFFFFFull) return MCX_E_INVALID;
    const uint32_t steps = (uint32_t)steps64;
    void *buf = nullptr, *sink = nullptr;
    if ((e = mcx::pool_alloc(&buf, sectors64 * 32, st)) != cudaSuccess) return MCX_E_OOM;
    if ((e = mcx::pool_alloc(&sink, 1024 * sizeof(uint32_t), st)) != cudaSuccess) {
        mcx::pool_free(buf, st);
        return MCX_E_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    e = cudaMemsetAsync(buf, 0x5A, sectors64 * 32, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        const int4 *b = static_cast<const int4 *>(buf);
        uint32_t *s = static_cast<uint32_t *>(sink);
        const uint32_t n = (uint32_t)sectors64;
        mcx::k_gather<<<grid, mcx::GATHER_THREADS, 0, st>>>(b, n, steps < 64 ? steps : 64, dependent, 1u, s);  // warm
        cudaEventRecord(e0, st);
        mcx::k_gather<<<grid, mcx::GATHER_THREADS, 0, st>>>(b, n, steps, dependent, 2u, s);
        cudaEventRecord(e1, st);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    mcx::pool_free(sink, st);
    mcx::pool_free(buf, st);
    if (e != cudaSuccess) return MCX_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MCX_E_CUDA;
    *sectors_per_second = ms > 0.0f ? (double)threads * (double)steps / ((double)ms * 1e-3) : 0.0;
    return MCX_OK;
}

}  // extern "C"
