/*
 * gmcs_diag.h -- diagnostics beside the particle-update library (libgmcs_diag.so).
 *
 * Not part of the particle-update ABI of gmcs.h: calibration measurements that
 * the benchmark takes to put the lookup passes' rates in context. The paper has
 * no counterpart. Status codes are those of gmcs.h.
 */
#ifndef GMCS_DIAG_H
#define GMCS_DIAG_H

#include <stdint.h>

#include "gmcs.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * The rate (GB/s, into *gbs) of random rec_bytes-sized (16 or 32) record reads
 * from a device buffer of buffer_bytes, with the loads of the lookup pass (one
 * 256-bit load per 32-byte record, one 128-bit load per 16-byte record) -- with
 * a buffer that fits L2 (126 MB), the ceiling for lookups whose cells stay in L2.
 * Allocates and frees the buffer; runs on cuda_stream and synchronises it.
 * Errors: GMCS_E_INVALID (rec_bytes not 16 or 32, buffer under one record),
 * GMCS_E_OOM, GMCS_E_CUDA.
 */
int gmcs_probe_gather(uint64_t buffer_bytes, int rec_bytes, void* cuda_stream, double* gbs);

/*
 * The device's FP32 FMA rate (TFLOP/s, an FMA counted as 2 flops, into *tflops):
 * eight independent fmaf chains per thread on sm_count x 8 CTAs of 256 threads,
 * best of five launches; *sm_count (may be NULL) receives the multiprocessor count
 * read from the device. Runs on cuda_stream and synchronises it.
 * Errors: GMCS_E_INVALID, GMCS_E_OOM, GMCS_E_CUDA.
 */
int gmcs_probe_ffma(void* cuda_stream, double* tflops, int* sm_count);

#ifdef __cplusplus
}
#endif

#endif /* GMCS_DIAG_H */
