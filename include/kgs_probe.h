/*
 * kgs_probe.h -- measurement kernels of libkgs (no counterpart in the paper).
 *
 * The DP-AVF2 colour passes in float64 are bound by the FP64 pipe of the B300,
 * whose rate the measured-peaks file does not give.  This probe measures it
 * (and the FP32 rate) the way a roofline denominator is usually taken: many
 * independent fused multiply-add chains per thread, enough CTAs to fill every
 * SM, timed with CUDA events on the given stream.  The other entry points
 * expose the float64 neighbour sums and Psi weight of the colour passes so
 * that tests can check them against exact arithmetic.
 */
#ifndef KGS_PROBE_H
#define KGS_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Run `iters` iterations of 8 independent FMA chains in every thread of a grid
 * of 148 * blocks_per_sm CTAs x 256 threads, in float64 (precision 64) or
 * float32 (precision 32), on the current device and `stream` (cudaStream_t as
 * void*, NULL = legacy default).  Writes the elapsed milliseconds and the FMA
 * rate in FMA/s (one FMA = 2 flops).  Synchronises the stream.
 * Returns 0, -1 for a bad argument (iters < 1, blocks_per_sm < 1 or > 64,
 * precision not 32/64, NULL outputs) or -4 if a CUDA call failed. */
int kgs_probe_fma_rate(int precision, int64_t iters, int blocks_per_sm, void* stream,
                       double* elapsed_ms, double* fma_per_s);

/* The float64 neighbour sums of the colour passes on n rows of k values
 * (k = 2, 4 or 6, the 2d neighbours of a point in 1, 2 or 3 dimensions):
 * x_host holds the rows one after another (n * k doubles, row-major).
 * sum_host receives each row's sum S and scaled_host beta * S as the passes
 * form them (beta = the Psi neighbour weight; any double here).
 * exact_host (may be NULL) receives per row bit 0 = S was formed in the exact
 * integer accumulator (then it is the correctly rounded sum of the row) and
 * bit 1 = beta S was (then it is beta times the exact sum, rounded once);
 * where a bit is 0 the left-to-right float64 sum (times beta, rounded) was
 * taken: an infinite or NaN value, a nonzero value more than 31
 * binades below the row's largest, a zero or subnormal beta, or a result
 * outside the normal range.  A row whose entry points disagreed with these
 * halves reads -1.  Host buffers are the caller's; the call copies through
 * device memory on the current device and `stream` and synchronises it.
 * Returns 0, -1 for a bad argument (k not 2, 4 or 6, n < 0, a NULL input or
 * output other than exact_host with n > 0), -3 if device memory could not
 * be allocated or -4 if a CUDA call failed. */
int kgs_probe_nsum(int k, int64_t n, const double* x_host, double beta, double* sum_host,
                   double* scaled_host, int32_t* exact_host, void* stream);

/* The weight w = 1 / (1 + r^2) of the colour passes' float64 Psi update for
 * n values r_host[i], written to w_host[i] (host buffers, the caller's; the
 * call copies through device memory on the current device and `stream` and
 * synchronises it).  Returns 0, -1 for a bad argument (n < 0, NULL buffers
 * with n > 0), -3 if device memory could not be allocated or -4 if a CUDA
 * call failed. */
int kgs_probe_psi_weight(int64_t n, const double* r_host, double* w_host, void* stream);

/* Index checks (the stand-in for a memory checker, which this build does not
 * rely on).  The library built with -DKGS_DEBUG_BOUNDS (libkgs_debug.so)
 * checks the indices of the colour-pass, streamed-plane and batch kernels
 * before every access; an index out of range sets a flag bit on the device
 * and the access is skipped (no trap).  This call synchronises the current
 * device, writes the OR of the flag bits set since the last call to *flags
 * (1 colour-pass index, 2 streamed-plane shared-memory index, 4
 * streamed-plane store, 8 batch index) and clears them.  Returns 1 in the
 * checking build, 0 in the normal one (where *flags is always 0), -1 for a
 * NULL flags or -4 if a CUDA call failed. */
int kgs_debug_bounds(uint32_t* flags);

/* The side list of the float32 3D two-steps-per-launch kernel
 * (KGS_OPT_KERNEL 8) for an N^3 grid, as the host builds it (no device
 * needed): the points beyond a tile's 32 colour columns that its first three
 * colour passes update, per tile kind (0: 23-row tiles, 1: the grid's last,
 * shorter row of tiles) and plane parity q.  out receives 2 x 2 x 96 entries
 * (kind-major, then q, then the list index), each staged row | staged column
 * << 5 | (passes - 1) << 11 | 0x8000 (staged row = tile row + 4, staged
 * column = colour column + 2) or 0 past the list's end, then the 2 x 2 list
 * lengths.  cap: uint16 entries at out.  Returns the entries written (388),
 * -1 for a bad argument (N not even or < 4, out NULL, cap < 388) or -2 if
 * the grid's regions break the kernel's thread layout (then the kernel is
 * not used for it). */
int kgs_stream2_side_list(int64_t N, uint16_t* out, int64_t cap);

#ifdef __cplusplus
}
#endif

#endif /* KGS_PROBE_H */
