/*
 * stfd_profile.h -- diagnostics of libstfd: per-kernel timing with CUDA
 * events, a launch counter, and a DFMA throughput probe. The paper reports
 * wall-clock only (Sec. 5, Tables 4-6 and Fig. 3); these calls exist so that
 * a caller can attribute the time of a solve to the kernels of Algorithm 1,
 * the system matvec and GMRES, and compare it with the FP64 peak of the GPU
 * it runs on. Nothing here changes results.
 */
#ifndef STFD_PROFILE_H
#define STFD_PROFILE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Turn per-launch event timing on (1) or off (0). While on, every kernel
 * launch of the library is bracketed by two cudaEvents recorded on the
 * stream it is launched on. Off by default. Returns STFD_OK. */
int stfd_profile_enable(int on);

/* Drop all timing records (synchronises on their events first). */
int stfd_profile_reset(void);

/* Number of distinct kernels with records; synchronises on pending events. */
int stfd_profile_count(void);

/* Record `idx` (0 <= idx < count): kernel name (NUL-terminated, truncated to
 * name_cap), launches, total device milliseconds, and the algorithmic FLOPs
 * and bytes (minimum HBM traffic: each input read once, each output written
 * once) summed over its launches. Any output pointer may be NULL. Returns
 * STFD_ERR_ARG for a bad index. */
int stfd_profile_get(int idx, char* name, int name_cap, long long* launches, double* ms,
                     double* flops, double* bytes);

/* Kernel launches issued by the library since it was loaded (always counted). */
long long stfd_launch_count(void);

/* FP64 FMA throughput of the current device in FLOP/s, measured with
 * independent DFMA chains on every SM (about 20 ms of device time). The
 * result is the denominator of an FP64-ALU roofline. Synchronous. */
int stfd_probe_fp64_peak(double* flops_per_s, void* stream);

/* Measured rate of 32 x 32 -> 64-bit integer multiply-adds (mad.wide.s32, eight
 * independent chains per thread, all SMs), in operations per second: the
 * ceiling of the integer-limb band products (STFD_OP_FX64), which need three
 * per tap. Synchronous; allocates a small buffer. */
int stfd_probe_imad_wide_peak(double* ops_per_s, void* stream);

/* Failure-detection self-test of the bounded device waits used by the
 * tensor-core kernels: one thread initialises an mbarrier that nothing ever
 * arrives on and waits on it for at most `max_iters` polls; when the wait gives
 * up it sets the same device status flag the tensor-core kernels set and
 * returns (no tensor core, tensor memory or other thread is involved). Read
 * the flag with stfd_device_status(), which then reports STFD_ERR_TIMEOUT and
 * clears it. 1 <= max_iters <= 1e6. Synchronous. */
int stfd_probe_bounded_wait(int max_iters, void* stream);

/* Self-test of the FP64 <-> double-float conversions that the double-float
 * and tensor-core kernels use at their FP64 inputs and outputs (built from
 * the IEEE 754 bit fields, off the FP64 pipe). For i < n, all device
 * pointers: pairs[2i], pairs[2i+1] = the double-float (h, l) of x[i];
 * back[i] = that pair converted back to FP64; f[i] = x[i] rounded to FP32;
 * fback[i] = f[i] converted back to FP64. n >= 0. Stream-ordered. */
int stfd_probe_convert(const double* x, long long n, float* pairs, double* back, float* f, double* fback,
                       void* stream);

#ifdef __cplusplus
}
#endif
#endif /* STFD_PROFILE_H */
