/*
 * lap_probe.h - measurement aid of the benchmark, not a step of the method and
 * not part of the method's library (built separately as liblap_probe.so).
 *
 * lap_probe_random_rw launches `blocks` x 256 threads on `cuda_stream` (NULL:
 * the legacy default stream); each thread does `rounds` rounds of 4
 * independent single-byte read-then-write pairs at addresses in [0, bytes) of
 * `device_buf` drawn from a SplitMix64 hash of (salt, thread, round), so
 * blocks * 256 * rounds * 4 pairs per launch.  This is the memory pattern of
 * one Wilson step of the 1-byte-state sampler (one random state-byte read, one
 * random state-byte write) without its dependent chain; timing the launch
 * (CUDA events on the same stream) gives the ceiling that pattern reaches on
 * the device.
 *
 * device_buf: caller-owned device memory of `bytes` bytes, which the probe
 * modifies (every byte it touches is incremented).  Returns
 * LAP_PROBE_ERR_INVALID_ARG for a NULL buffer, bytes == 0 or blocks == 0,
 * LAP_PROBE_ERR_CUDA if the launch fails, LAP_PROBE_OK otherwise
 * (asynchronous).
 */
#ifndef LAP_PROBE_H_
#define LAP_PROBE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { LAP_PROBE_OK = 0, LAP_PROBE_ERR_INVALID_ARG = 1, LAP_PROBE_ERR_CUDA = 10 };

int lap_probe_random_rw(void *device_buf, uint64_t bytes, uint32_t blocks, uint32_t rounds, uint64_t salt,
                        void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LAP_PROBE_H_ */
