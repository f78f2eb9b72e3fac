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

/* rad_probe_loop - the accumulate kernel's update loop with parts removed, on
 * the current device (timing only: the arithmetic is real, the results are
 * discarded).  One 256-particle tile of synthetic records in shared memory is
 * swept by 256-thread blocks, 2 per SM, each warp holding four 16-frequency
 * MMA blocks, with no stage 1, barrier or epilogue.  Per mode m, out[2 m] =
 * MUFU sin/cos lane-operations per SM clock and out[2 m + 1] = the effective
 * clock (MHz):
 *   m = 0  the variant-8 update: phase reduction, TF32 hi/lo split, 4 mma.sync;
 *   m = 1  without the split (the raw sin/cos bits into the same 4 MMAs);
 *   m = 2  the split without the MMAs (its results folded by XOR);
 *   m = 3  neither (sin/cos consumed by 2 packed FMAs);
 *   m = 4  the variant-9 update (phase cross terms by one more mma.sync).
 * out: host array of n_out >= 10 doubles.  Returns 0, or a CUDA error code.
 * Allocates a few MB of device memory for the duration of the call. */
int rad_probe_loop(double* out, int n_out);

#ifdef __cplusplus
}
#endif

#endif /* RAD_PROBE_H */
