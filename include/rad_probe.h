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

/* rad_probe_tensor - tensor-pipe probes on the current device, into out[0..7]:
 *   [0] legacy mma.sync m16n8k8 TF32: multiply-adds per SM clock;
 *   [1..4] SM clocks per tcgen05.mma kind::tf32 (M = 128, K = 8, A in tensor
 *          memory, B in shared memory) at N = 16, 64, 128, 256;
 *   [5], [6] the same for kind::f16 (K = 16) at N = 16 and 256 (-1 if an MMA
 *          wait ran out);
 *   [7] the effective clock (MHz) of the mma.sync probe.
 * Each tcgen05 probe runs one single-warp CTA per SM holding all 512 tensor-
 * memory columns.  out: host array of n_out >= 8 doubles.  Returns 0, or a CUDA
 * error code.  Allocates a few MB of device memory for the duration of the call. */
int rad_probe_tensor(double* out, int n_out);

#ifdef __cplusplus
}
#endif

#endif /* RAD_PROBE_H */
