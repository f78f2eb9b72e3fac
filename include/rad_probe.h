/*
 * rad_probe.h - pipe-throughput probe of the GPU the radiation library runs on
 * (roofline denominators of the mixed-precision kernel).  The paper has no
 * counterpart; it reports no performance figures.
 */
#ifndef RAD_PROBE_H
#define RAD_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* rad_probe_peaks - run the probes on the current device and write, per probe,
 * lane-operations per SM clock (from the SM cycle counter) and the effective
 * clock in MHz (cycles / wall time) into out[0..15]:
 *   [0,1] FP32 FMA   [2,3] packed FP32x2 FMA   [4,5] MUFU sin/cos   [6,7] FP64 FMA
 *   [8,9] float round-to-integer   [10,11] f64<->f32 conversions
 *   [12,13] MUFU with 8 packed FMAs per 4 MUFU   [14,15] with 16 per 4.
 * out: host array of n_out >= 16 doubles.  Returns 0, or a CUDA error code.
 * Allocates a few MB of device memory for the duration of the call. */
int rad_probe_peaks(double* out, int n_out);

#ifdef __cplusplus
}
#endif

#endif /* RAD_PROBE_H */
