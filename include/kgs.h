/*
 * kgs.h -- C ABI of libkgs: the DP-AVF2 checkerboard solver for the periodic
 * Klein-Gordon-Schroedinger equations on a B300 GPU (sm_103a).
 *
 * The method (arXiv 2502.09537):
 *   i psi_t + (kappa1/2) Lap psi + gamma u psi = 0,
 *   u_tt - kappa2 Lap u + mu^2 u - gamma |psi|^2 = 0            (Eq. kgs, Sec. 1)
 * on the periodic box [-L/2, L/2)^d, d in {1,2,3}, discretised by central
 * differences on N points per direction, h = L/N (Sec. 2, Eq. kgs-semi), and
 * advanced by DP-AVF2 = Phi*_{tau/2} o Phi_{tau/2} (Eq. dp-comp): the explicit
 * pointwise base update of Eq. scheme1 and its adjoint (Eq. dp-avf-kj-adj),
 * swept in the checkerboard order of Sec. 4.2 / Algorithm 3 (red = points whose
 * 1-based index sum is odd; base half red then black, adjoint half black then
 * red).  The scheme conserves the discrete energy E_h exactly (Thm. 3.1).
 *
 * State layout seen by callers: four float64 arrays P = Re psi, Q = Im psi,
 * U = u, V = u_t, each of N^d elements in C order with shape (N,)*d and index
 * [ix][iy][iz] (z fastest), the paper's linear index i = (j-1)N + k (Sec. 2).
 * Grid point [ix][iy][iz] sits at (-L/2 + ix h, -L/2 + iy h, -L/2 + iz h).
 *
 * Ownership: the library owns every device buffer of a handle (allocated in
 * kgs_create*, freed in kgs_destroy).  Caller buffers passed to kgs_set_state /
 * kgs_get_state are never retained.  The order in which a handle keeps its
 * state on the device is the library's own (each colour's points contiguous)
 * and never seen by callers, who always exchange the layout above.
 *
 * Streams: every `stream` argument is a cudaStream_t passed as void*; NULL is
 * the legacy default stream.  Calls that take device buffers are asynchronous
 * on that stream; calls that take host buffers or return host values
 * synchronise it before returning.  kgs_energy and kgs_mass run on the stream
 * of the handle's latest kgs_set_state / kgs_step call.
 *
 * Threading: a handle is not thread-safe; distinct handles are independent.
 * Errors: functions return KGS_OK (0) or a negative status.  kgs_last_error()
 * gives a message for the calling thread's most recent failure.  A CUDA error
 * inside a call is returned as KGS_ERR_CUDA and is also kept in the handle
 * (every later call on it returns KGS_ERR_CUDA until it is destroyed).
 */
#ifndef KGS_H
#define KGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define KGS_OK            0
#define KGS_ERR_ARG      -1  /* invalid argument (dim, L, parameters, NULL pointer, where) */
#define KGS_ERR_ODD_N    -2  /* N odd or N < 4: the periodic checkerboard needs even N */
#define KGS_ERR_OOM      -3  /* device allocation failed (or would take the handle past
                                  KGS_DEVICE_BUDGET: an environment variable, in bytes, read by
                                  kgs_create; it caps what one handle allocates -- its state and
                                  the buffers options add on first use -- so that the out-of-
                                  memory paths can be exercised without exhausting the device) */
#define KGS_ERR_CUDA     -4  /* a CUDA call failed (also: no usable device) */
#define KGS_ERR_STATE    -5  /* no state set yet */
#define KGS_ERR_TIMEOUT  -6  /* a bounded device wait ran out (a grid barrier of the persistent
                               order launch, or a dependency wait of the wave kernel or of the
                               lexicographic sweep, did not complete within 2 s); the
                               handle's state is lost and every later call on the handle
                               returns this status */
#define KGS_ERR_RANGE    -7  /* size beyond what the call supports */

/* memory kind of caller buffers */
#define KGS_HOST   0
#define KGS_DEVICE 1
#define KGS_HOST_ASYNC 2  /* host memory, queued on the stream without waiting (see kgs_set_state) */

/* state precision (kgs_create_ex) */
#define KGS_FP64 64  /* state and arithmetic in float64 */
#define KGS_FP32 32  /* state and arithmetic in float32; invariants in float64 */

/* options (kgs_set_option) */
#define KGS_OPT_KERNEL   1  /* 0 auto, 1 one launch per colour pass, 2 shared-memory resident,
                               3 temporally blocked tiles (dim 2, 3; allocates a second state
                               buffer of the same size on first use), 4 persistent grid-stride
                               colour passes, 5 colour passes pipelined in axis-0 slabs through
                               L2 (dim 2, 3; see KGS_OPT_SLAB_PLANES), 6 wave kernel: a step's
                               two colour passes in one cooperative launch whose CTAs take
                               slab chunks in a dependency-safe order (dim 2, 3, N >= 64;
                               KGS_OPT_SLAB_PLANES sets the slab, 0 = about 4 MB of state;
                               grids it does not fit run the plain passes), 7 streamed planes:
                               a step's two colour passes in one launch that walks axis 0 with
                               every plane of a 29 x 64 tile staged by a TMA tensor load
                               (float32 state, dim 3, N a multiple of 64 up to 1024; allocates
                               two packed copies of the state, about 2.2 GB each at N = 512, on
                               first use; other grids run the plain passes), 8 streamed planes,
                               two steps per launch: a step pair's four colour passes chained
                               plane by plane in one launch over 23 x 64 tiles staged with a
                               four-row halo (temporal depth 2: one read and one write of the
                               state per two steps; an odd step count ends with one launch of
                               7; same grids and buffers as 7).  Auto picks 2 for grids that fit
                               one CTA's shared memory, 8 where it applies and N >= 128, 1
                               otherwise.  All give bitwise the same state. */
#define KGS_OPT_GRAPH    2  /* 0 off, 1 replay colour passes from a CUDA graph (default 1) */
#define KGS_OPT_THREADS  3  /* CTA size of the colour-pass kernels: 128, 256 (default), 512 */
#define KGS_OPT_PPT      4  /* points of one colour per thread in those kernels: 1 only (2 was
                               measured no faster: the FP64 pipe, not latency, binds) */
#define KGS_OPT_TILE_T1      5  /* tile kernel: tile extent along axis 1 (3D) */
#define KGS_OPT_TILE_T2      6  /* tile kernel: tile extent along the last axis (even) */
#define KGS_OPT_TILE_LX      7  /* tile kernel: axis-0 planes per CTA */
#define KGS_OPT_TILE_PASSES  8  /* tile kernel: colour passes per launch (= halo width), 1..8 */
#define KGS_OPT_TILE_THREADS 9  /* tile kernel: threads per CTA (64, 128, 256, 512, 1024) */
#define KGS_OPT_ORDER_MODE  11  /* update orders (kgs_set_order): 0 auto (default: mode 4 or 3,
                                   or mode 1 if the second state buffer cannot be allocated), 1 one
                                   launch per level on the handle's state layout (a step captured
                                   in a CUDA graph), 2 every level of a step in one cooperative
                                   persistent launch with a grid barrier after each level
                                   (bounded: see KGS_ERR_TIMEOUT; kgs_step then waits for the
                                   device before returning), 3 one launch per level on a natural-
                                   order copy of the state (a second state buffer, allocated on
                                   first use; each kgs_step call converts into it and back), 4 for
                                   the lexicographic order or its reverse in 2D with N a multiple
                                   of 32: on that copy, a doacross sweep in one cooperative launch
                                   per half step -- one warp per strip of 32 rows, its lanes one
                                   column apart, each strip trailing the one before it (waits
                                   bounded: see KGS_ERR_TIMEOUT; other orders and grids: as 3).
                                   Auto takes 4 where it applies.  All compute bitwise the same
                                   state. */
#define KGS_OPT_TEST_BARRIER_STALL 12  /* test hook: n > 0 makes every grid barrier of the
                                   persistent order launch wait for n CTAs that do not exist, and
                                   every dependency wait of the wave kernel and of the
                                   lexicographic sweep for n chunks or steps that do not
                                   exist, and makes the streamed-plane kernel wait once on a
                                   barrier that nothing completes, so they time out (after 2 s) and the handle reports
                                   KGS_ERR_TIMEOUT (kgs_step for the order launch, which waits for
                                   the device; the next synchronising call for the others);
                                   0 (default) off.  For testing the timeout path only. */
#define KGS_OPT_WAVE_LAG    13  /* wave kernel: slabs by which the red pass trails the black pass
                                   in the ticket order, 1 .. 64; 0 (default) = enough for the
                                   chunks in flight (2 + CTAs / (2 chunks per slab)) */
#define KGS_OPT_WAVE_CHUNK  14  /* wave kernel: points of a colour per chunk (rounded down to
                                   whole rows, at least one), 1 .. 2^24; 0 (default) = 2048 */
#define KGS_OPT_PDL         15  /* 1 (default): launch the one-per-pass colour passes (kernel 1)
                                   with programmatic dependent launch, each waiting in the kernel
                                   for the one before, so a pass's launch overlaps the previous
                                   pass's tail (+0.3% on the 2D FP64 workload); 0 plain launches.
                                   Bitwise the same state either way. */
#define KGS_OPT_STREAM_CHUNK 16 /* streamed-plane kernels (7, 8): C > 0: work items of C axis-0 planes
                                   of a tile, taken round-robin chunk by chunk, so that neighbouring
                                   tiles stream the same planes together (their shared halo rows
                                   then come from L2); 0 (default) = the fewest chunks per tile
                                   column, at least two, that fill 95% of the rounds of CTAs over
                                   the SMs (256 planes at N = 512 on 148 SMs for 7, 128 for 8);
                                   -1: each CTA takes a contiguous share of the (tile, plane)
                                   sequence instead.  Bitwise the same state. */
#define KGS_OPT_STREAM_PREFETCH 17 /* streamed-plane kernels (7, 8): planes beyond its shared-memory
                                   loads that a CTA also asks L2 to fetch ahead (TMA prefetch),
                                   0 .. 16; default 2.  Bitwise the same state. */
#define KGS_OPT_SLAB_PLANES 10  /* slab and wave kernels: axis-0 planes per slab, 1 .. N (the
                                   wave kernel takes the largest divisor of N not above it);
                                   0 (default) picks about a quarter of the L2 cache's bytes per
                                   slab for the slab kernel.  A step's
                                   black pass runs slab by slab and each slab's red pass follows
                                   the next slab's black pass, so the two passes reuse the state
                                   in L2 instead of reading it from HBM twice; every point sees
                                   the neighbour values of the two full passes (bitwise equal) */

typedef struct kgs_solver* kgs_handle;

/* Create a solver for dimension dim in {1,2,3}, N points per direction (even,
 * >= 4), period L > 0, finite kappa1, kappa2, mu, gamma (either sign) and a
 * finite, nonzero time step tau (negative tau runs the scheme backwards,
 * Eq. dp-comp being symmetric).  FP64 state on the current device.
 * Allocates 2 * N^d * 16 bytes of state plus N^d * 8 bytes of staging and a
 * few KB of reduction scratch.  Returns NULL on error (see kgs_last_error). */
kgs_handle kgs_create(int dim, int64_t N, double L, double kappa1, double kappa2,
                      double mu, double gamma, double tau);

/* As kgs_create, with precision KGS_FP64 or KGS_FP32 and a CUDA device index
 * (-1 = the current device).  FP32 halves the state bytes. */
kgs_handle kgs_create_ex(int dim, int64_t N, double L, double kappa1, double kappa2,
                         double mu, double gamma, double tau, int precision, int device);

/* Copy a state in: four float64 arrays of N^d elements each (layout above),
 * host memory (where = KGS_HOST; pinned or pageable; returns after the copy)
 * or device memory of the handle's device (where = KGS_DEVICE; asynchronous on
 * stream; the buffers must stay valid until the stream reaches this point).
 * where = KGS_HOST_ASYNC: host memory, copied asynchronously on stream like
 * device memory (the buffers must stay valid and unchanged until the stream
 * reaches this point; pinned memory lets the copies overlap other streams'
 * work, pageable memory makes them synchronous).  The handle's one staging
 * buffer carries every host copy in and out, so host copies of one handle
 * must be ordered with each other and with its kgs_step calls (one stream,
 * or events).  FP32 handles round each value to float32. */
int kgs_set_state(kgs_handle h, const double* P, const double* Q, const double* U,
                  const double* V, int where, void* stream);

/* Copy the state out as four float64 arrays (FP32 state is widened exactly).
 * Host buffers are filled when the call returns; device buffers (and host
 * buffers with where = KGS_HOST_ASYNC) are written asynchronously on stream,
 * with the ordering rules of kgs_set_state. */
int kgs_get_state(kgs_handle h, double* P, double* Q, double* U, double* V,
                  int where, void* stream);

/* Advance the state by nsteps >= 0 full DP-AVF2 steps of size tau (Eq. dp-comp
 * in the checkerboard order of Algorithm 3, or the order set by
 * kgs_set_order), asynchronously on stream.  On completion the state is at a
 * step boundary; kgs_step(a) then kgs_step(b) gives bitwise the result of
 * kgs_step(a + b). */
int kgs_step(kgs_handle h, int64_t nsteps, void* stream);

/* ---- update orders (Sec. 3, Eqs. LapP, order1, order2; Algorithms 1-2) ----
 * Any order of the grid points defines a DP-AVF scheme: in a point's update
 * the neighbours that come earlier in the order enter at the new level and
 * the later ones at the old level (the S/W/E/N superscripts of Eq. LapP).
 * DP-AVF2 visits the points in the order in its base half and in the reverse
 * order in its adjoint half (Algorithm 1), in place.  The checkerboard of
 * Algorithm 3 is the default; Eq. order1 is the lexicographic order (C order
 * of the linear index), Algorithm 2 a block-splitting order.
 *
 * An order is a permutation of the linear indices 0 .. N^d - 1 of the grid
 * (C order: index = (i0 N + i1) N + i2, last axis fastest).  It runs on the
 * device as a level schedule: the level of a point is one more than the
 * largest level of its neighbours that precede it in the order (0 if none);
 * points of one level are never neighbours and are updated in parallel, the
 * levels in increasing order in the base half and in decreasing order in the
 * adjoint half.  This gives every point exactly the neighbour values of the
 * serial order, so the result does not depend on how points of one level
 * are ordered.  The checkerboard has 2 levels, the lexicographic order
 * 1 + d (N - 1) (its anti-diagonal wavefronts).
 *
 * kgs_order_schedule: the levels of `order` (N^d int64, host, the caller's)
 * written to level[0 .. N^d) (host, by linear index) and their count to
 * *nlevels.  Host only: needs no device.  Returns KGS_OK, KGS_ERR_ARG (NULL
 * argument, dim not 1-3, or order not a permutation), KGS_ERR_ODD_N,
 * KGS_ERR_RANGE (N^d beyond what kgs_create takes) or KGS_ERR_OOM (host
 * memory).
 *
 * kgs_set_order: make `order` (N^d int64, host; copied) the handle's update
 * order from the next kgs_step on; NULL restores the checkerboard.  The
 * handle keeps the points sorted by level on the device (8 bytes per point);
 * the colour-pass kernel options apply to the checkerboard only and
 * KGS_OPT_ORDER_MODE to the other orders.  Waits for
 * the device to finish queued work first.  Returns KGS_OK, KGS_ERR_ARG (not
 * a permutation; the handle's order is unchanged), KGS_ERR_OOM (host or
 * device memory) or KGS_ERR_CUDA.
 *
 * kgs_set_orders: one update order for Psi (order_psi) and another for (U,V)
 * (order_uv), both N^d int64 on the host, copied (the remark after Eq.
 * dp-avf-kj-adj: the variables may follow different orders).  A point's Psi
 * update reads U only at that point and its (U,V) update reads Psi only at
 * that point, so Algorithm 1's per-point procedure over one order is two whole
 * sweeps, and with two orders each half step is: base -- Psi over order_psi
 * (with U^n), then (U,V) over order_uv (with |Psi^{n+1}|^2); adjoint --
 * (U,V) over order_uv reversed, then Psi over order_psi reversed (with
 * U^{n+1}).  Equal orders give exactly kgs_set_order's scheme.  These orders
 * run as per-level launches (KGS_OPT_ORDER_MODE 1 or 3; modes 2 and 4 apply
 * to one common order only).  Both pointers are required; kgs_set_order
 * (also with NULL) returns to one order.  Returns as kgs_set_order; on
 * KGS_ERR_ARG for order_uv nothing changes.
 *
 * kgs_order_levels: the number of level launches per half step of the
 * handle's current order(s) (2 for the checkerboard; with two orders, the
 * sum of their levels). */
int kgs_order_schedule(int dim, int64_t N, const int64_t* order, int32_t* level, int64_t* nlevels);
int kgs_set_order(kgs_handle h, const int64_t* order);
int kgs_set_orders(kgs_handle h, const int64_t* order_psi, const int64_t* order_uv);
int kgs_order_levels(kgs_handle h, int64_t* nlevels);

/* Discrete invariants of the current state, computed on the device in float64
 * with compensated final summation, returned in host memory (synchronises
 * stream):
 *   out[0] = E_h = h^d sum [1/2 (kappa1 |grad_h psi|^2 + kappa2 |grad_h u|^2
 *                  + v^2 + mu^2 u^2) - gamma |psi|^2 u]   (Sec. 2, Eq. ene-origin;
 *            grad_h the forward difference, via summation by parts)
 *   out[1] = h^d sum of the absolute values of those five terms (a scale for
 *            relative energy errors: E_h has no fixed sign)
 *   out[2] = mass h^d sum |psi|^2 (the discrete norm of Sec. 2; the scheme does
 *            not conserve it -- a diagnostic only). */
int kgs_invariants(kgs_handle h, double* out3, void* stream);

/* E_h and the mass alone (out[0] and out[2] of kgs_invariants). */
int kgs_energy(kgs_handle h, double* E);
int kgs_mass(kgs_handle h, double* M);

/* Change the time step (finite, nonzero; either sign).  Takes effect for the
 * next kgs_step. */
int kgs_set_tau(kgs_handle h, double tau);

/* Tuning options (KGS_OPT_*); values out of range return KGS_ERR_ARG.  None
 * changes results: every kernel variant computes bitwise the same state (the
 * test hook KGS_OPT_TEST_BARRIER_STALL makes stepping fail on purpose). */
int kgs_set_option(kgs_handle h, int option, int64_t value);

/* Number of kernels this handle has launched so far (graph replays count
 * each kernel node).  For benchmarks. */
int64_t kgs_launch_count(kgs_handle h);

/* Free every device buffer of the handle.  NULL is ignored. */
void kgs_destroy(kgs_handle h);

/* Static message for a status code. */
const char* kgs_strerror(int status);

/* Message of the calling thread's most recent error ("" if none). */
const char* kgs_last_error(void);

/* Status of the calling thread's most recent failed call (KGS_OK if none);
 * the way to learn why kgs_create / kgs_create_ex returned NULL. */
int kgs_last_status(void);

/* ---- batches of independent instances -----------------------------------
 * Many KGS problems of different dimensions, sizes, parameters and precisions
 * stepped together on one device, each bitwise as if stepped alone (the same
 * pointwise updates of Eqs. scheme1 / dp-avf-kj-adj in the checkerboard order
 * of Algorithm 3).  One launch per colour pass and precision covers every
 * instance (a persistent grid over a work list of 256-point chunks); the
 * launches of a step call are captured in a CUDA graph and replayed while the
 * instance set and step counts stay the same.  The batch owns one device arena
 * of a fixed capacity (the memory budget); instances are placed in it first
 * fit and their space is returned by kgs_batch_remove. */
typedef struct kgs_batch* kgs_batch_handle;

#define KGS_BATCH_OPT_CTAS_PER_SM 1  /* persistent CTAs per SM, 1..32 (default 8), every list */
#define KGS_BATCH_OPT_GRAPH       2  /* 0 off, 1 capture step calls in a CUDA graph (default 1) */
/* Persistent CTAs per SM of one list of instances -- one precision and
 * dimension, whose passes share a launch: option KGS_BATCH_OPT_CTAS_LIST +
 * 3 p + (dim - 1), p = 0 for FP64 and 1 for FP32, value 1..32, or 0 to follow
 * KGS_BATCH_OPT_CTAS_PER_SM again (which also resets every list). */
#define KGS_BATCH_OPT_CTAS_LIST   16
/* 1: each kgs_batch_step / step_each call is one persistent cooperative launch
 * (in the CUDA graph, when graphs are on) that runs every colour pass of every
 * instance, both precisions and every dimension, with a bounded grid barrier
 * between passes (a wait past 2 s makes the batch report KGS_ERR_TIMEOUT from
 * its next call on); CTAs per SM: KGS_BATCH_OPT_CTAS_PER_SM, at most what fits.
 * Batches with an instance of 2^31 points or more take the per-pass launches.
 * 0 (default): one launch per colour pass, precision, dimension and mode, the
 * lists on their own streams.  Bitwise the same states either way. */
#define KGS_BATCH_OPT_PERSISTENT  3
/* test hook: n > 0 makes the persistent launch's grid barrier wait for n CTAs
 * that do not exist, so that it times out (KGS_ERR_TIMEOUT); 0 (default) off. */
#define KGS_BATCH_OPT_TEST_STALL  4

/* Create a batch on `device` (-1 = current) with an arena of capacity_bytes
 * (>= 4096).  NULL on error (kgs_last_status / kgs_last_error). */
kgs_batch_handle kgs_batch_create(int device, int64_t capacity_bytes);

/* Add an instance (arguments as kgs_create_ex; precision KGS_FP64 or
 * KGS_FP32).  Returns its index (>= 0; indices of removed instances are
 * reused) or a negative status: KGS_ERR_OOM when no free arena range holds its
 * 2 * N^d * 16 (FP64) or 8 (FP32) bytes. */
int64_t kgs_batch_add(kgs_batch_handle b, int dim, int64_t N, double L, double kappa1,
                      double kappa2, double mu, double gamma, double tau, int precision);

/* Remove an instance and return its arena range. */
int kgs_batch_remove(kgs_batch_handle b, int64_t id);

/* Largest free contiguous arena range in bytes (negative status on error). */
int64_t kgs_batch_free_bytes(kgs_batch_handle b);

/* State in / out of one instance; arguments and behaviour as kgs_set_state /
 * kgs_get_state with KGS_HOST or KGS_DEVICE (host buffers use a temporary
 * device staging buffer; KGS_HOST_ASYNC is refused with KGS_ERR_ARG). */
int kgs_batch_set_state(kgs_batch_handle b, int64_t id, const double* P, const double* Q,
                        const double* U, const double* V, int where, void* stream);
int kgs_batch_get_state(kgs_batch_handle b, int64_t id, double* P, double* Q, double* U,
                        double* V, int where, void* stream);

/* Advance live instance i by nsteps[i] >= 0 full DP-AVF2 steps (array indexed
 * by instance index, entries of removed indices ignored), asynchronously on
 * stream.  Every stepped instance must have a state. */
int kgs_batch_step_each(kgs_batch_handle b, const int64_t* nsteps, void* stream);

/* Advance every live instance by nsteps. */
int kgs_batch_step(kgs_batch_handle b, int64_t nsteps, void* stream);

/* Invariants of one instance (as kgs_invariants; synchronises stream). */
int kgs_batch_invariants(kgs_batch_handle b, int64_t id, double* out3, void* stream);

int kgs_batch_set_option(kgs_batch_handle b, int option, int64_t value);
int64_t kgs_batch_launch_count(kgs_batch_handle b);

/* Free the arena and every device buffer of the batch.  NULL is ignored. */
void kgs_batch_destroy(kgs_batch_handle b);

/* ---- allocation-free invariants (no counterpart in the paper) ----------
 * The same three values as kgs_invariants (E_h, S_E, mass), for callers that
 * cannot allocate device memory where they need them: code whose GPU memory
 * is all owned by its own arena or budget, host threads that cannot afford
 * the implicit synchronisation of cudaMalloc, or callers that cannot create a
 * kgs handle (handle creation allocates).  No handle is involved and the call
 * allocates nothing: it reads the caller's state and writes the caller's
 * output, and keeps its reduction scratch in one fixed 192 KB array inside
 * libkgs that every GPU which loads the library holds until the process exits.
 *
 * P, Q, U, V: float64 device arrays of N^dim points in the layout above, on
 * the current device.  out3: float64 device array of 3, written
 * asynchronously on stream (cudaStream_t as void*, NULL = legacy default).
 * The grid may hold at most KGS_NOALLOC_MAX_POINTS points; larger grids are
 * rejected with KGS_ERR_RANGE before any work.  Invalid arguments return
 * KGS_ERR_ARG, CUDA failures KGS_ERR_CUDA (see kgs_last_error).
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  The address is kept per device and context: after a
 * cudaDeviceReset (a new context) the next call looks it up again, so make
 * that call outside a stream capture too.  All calls share the one scratch array: calls that can
 * run at the same time on the GPU (e.g. unordered streams) race and may return
 * wrong values; order them on one stream or with events. */
#define KGS_NOALLOC_MAX_POINTS 33554432  /* 8192 partial triples x 4096 points each */
int kgs_invariants_noalloc(int dim, int64_t N, double L, double kappa1, double kappa2,
                           double mu, double gamma, const double* P, const double* Q,
                           const double* U, const double* V, double* out3, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KGS_H */
