// Random-access probe (a measurement aid, not a step of the method): each
// thread performs rounds of independent single-byte read-then-write pairs at
// hashed addresses of a large device buffer -- the memory pattern of one
// Wilson step of the 1-byte-state samplers (read a node's state byte, write a
// state byte), without the dependent chain that limits a sampler lane.  The
// benchmark times it to measure the ceiling this pattern reaches on the
// device, the denominator its sampler throughput is compared with.  It is
// built into its own library (liblap_probe.so), apart from the method's.
#include <cstdint>

#include <cuda_runtime.h>

#include "lap_probe.h"

namespace {

// SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014; constants of Vigna's
// reference version).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr int kPairsPerRound = 4;

__global__ void __launch_bounds__(256) random_rw_kernel(uint8_t *buf, uint64_t bytes, uint32_t rounds, uint64_t salt)
{
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint32_t r = 0; r < rounds; ++r) {
        uint64_t a[kPairsPerRound];
#pragma unroll
        for (int j = 0; j < kPairsPerRound; ++j)
            a[j] = splitmix64(salt + t * 0x9E3779B97F4A7C15ull + (uint64_t)r * kPairsPerRound + (uint64_t)j) % bytes;
        uint32_t v[kPairsPerRound];
#pragma unroll
        for (int j = 0; j < kPairsPerRound; ++j) v[j] = buf[a[j]];
#pragma unroll
        for (int j = 0; j < kPairsPerRound; ++j) buf[a[j]] = (uint8_t)(v[j] + 1u);
    }
}

}  // namespace

extern "C" int lap_probe_random_rw(void *device_buf, uint64_t bytes, uint32_t blocks, uint32_t rounds,
                                          uint64_t salt, void *cuda_stream)
{
    if (!device_buf || bytes == 0 || blocks == 0) return LAP_PROBE_ERR_INVALID_ARG;
    if (rounds == 0) return LAP_PROBE_OK;
    random_rw_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(static_cast<uint8_t *>(device_buf),
                                                                               bytes, rounds, salt);
    return cudaGetLastError() == cudaSuccess ? LAP_PROBE_OK : LAP_PROBE_ERR_CUDA;
}
