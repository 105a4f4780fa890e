/*
 * libnglod measurement probes.  The paper has no counterpart: these kernels
 * measure the hardware ceilings that the benchmark's rooflines divide by --
 * the L2 and L1 read bandwidth that the feature gathers of Sec. 3.4 draw on,
 * and the FP32 FMA throughput of the CUDA-core decode.  Each call only
 * enqueues one kernel on the stream (a cudaStream_t passed as void*); the
 * caller times it with CUDA events and divides the bytes or flops the call
 * reports by that time.  Nothing is allocated; nothing synchronises.
 * Errors: NGLOD_ERR_INVALID_ARG for the cases named, NGLOD_ERR_CUDA if the
 * launch fails.
 */
#ifndef NGLOD_PROBE_H
#define NGLOD_PROBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Reads the device buffer buf (bytes long, 16-byte aligned, >= 16 bytes)
 * `passes` times with 16-byte loads cached in L2 only (ld.global.cg), every
 * block striding over the whole buffer; a buffer well below the L2's
 * capacity measures the L2 read bandwidth.  sink: one device word (written
 * only in a case that practically never occurs).  *h_bytes_read (nullable)
 * receives the bytes the kernel reads. */
int nglod_probe_l2_read(const void* buf, int64_t bytes, int passes, void* sink, int64_t* h_bytes_read,
                        void* stream);

/* Each block reads its own window of window_bytes (a multiple of 32 in
 * [64, 1 MiB], buf 32-byte aligned, bytes >= window_bytes) `passes` times
 * with 32-byte read-only loads (ld.global.nc, the gathers' form), so a window
 * that fits an SM's L1 measures the L1 read bandwidth.  Arguments otherwise
 * as nglod_probe_l2_read. */
int nglod_probe_l1_read(const void* buf, int64_t bytes, int64_t window_bytes, int passes, void* sink,
                        int64_t* h_bytes_read, void* stream);

/* FP32 fused multiply-adds: 8 SMs-worth of 256-thread blocks per SM, each
 * thread running 8 independent chains for 16 x iters steps (iters >= 1).
 * *h_flops (nullable) receives 2 x the FMAs executed. */
int nglod_probe_ffma(int64_t iters, void* sink, int64_t* h_flops, void* stream);

/* The number of SMs of the current device (the count the library's
 * persistent launches are sized by). */
int nglod_device_sms(int* h_sms);

#ifdef __cplusplus
}
#endif

#endif /* NGLOD_PROBE_H */
