/*
 * rc_probe.h -- measurement aids for the rooflines of the raycaster's gather
 * kernels. They are not part of the raycasting interface (include/rc.h) and
 * the paper has no counterpart: they only read memory at the highest rate a
 * plain kernel reaches, so that a march's achieved bytes per second can be set
 * against a measured peak of the memory level that serves its loads.
 *
 * Both calls launch one kernel on `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream) of the current device and return its launch status
 * (a cudaError_t value, 0 on success). Time them with events on that stream.
 * buf: device memory, 16-byte aligned; bytes: a multiple of 16; reps >= 1.
 * The kernels write nothing a caller can observe.
 */
#ifndef RC_PROBE_H
#define RC_PROBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* L2 read rate: a grid of 8 CTAs per SM reads buf reps times with 16-byte
 * loads that bypass L1 (ld.global.cg), each warp 512 contiguous bytes per
 * load. With bytes below the L2 size (129 MB on GB300) and well above L1's,
 * bytes * reps / time is the L2-to-SM read bandwidth. */
int rc_probe_read_l2(const void *buf, size_t bytes, int reps, void *cuda_stream);

/* L1 read rate: every CTA (4 per SM, 256 threads) reads the same small
 * buffer reps times with 16-byte loads through the read-only data path the
 * march's gathers use (ld.global.nc), each warp 512 contiguous bytes per load.
 * With bytes of a few tens of KB the buffer stays in each SM's L1 after the
 * first pass, and (CTAs * reps * bytes) / time is the L1 load bandwidth of the
 * whole GPU for fully coalesced 16-byte loads. At most 64 KB. */
int rc_probe_read_l1(const void *buf, size_t bytes, int reps, void *cuda_stream);

/* Bytes one rc_probe_read_l1 launch reads (CTAs * reps * bytes) on the
 * current device, or 0 when the device cannot be queried. */
size_t rc_probe_l1_bytes(size_t bytes, int reps);

#ifdef __cplusplus
}
#endif

#endif /* RC_PROBE_H */
