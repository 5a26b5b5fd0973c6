// kgs_internal.h -- declarations shared by the .cu files of libkgs (not public).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

#include "kgs_point.cuh"

namespace kgs {

// Geometry of one periodic grid: N points per direction, M = N^dim points.
struct Grid {
    int dim;
    int64_t N;
    int64_t M;
    int threads = 256;  // CTA size of the colour-pass kernels (128, 256 or 512)
    bool persistent = false;  // grid-stride persistent colour passes
    // axis-0 planes a colour pass covers: [plane0, plane0 + planes); planes = 0
    // means all N (one-launch-per-pass kernels only; 2D and 3D)
    int64_t plane0 = 0, planes = 0;
    bool split = false;  // state in the colour-split layout (below)
    bool pdl = false;    // launch with programmatic dependent launch (slab schedule)
    bool pdl_wait = false;  // ... and make black passes wait for their predecessor too
};

// Colour-split state layout (a handle's state): the points of even coordinate
// sum first, then those of odd coordinate sum, each colour in natural (C)
// order; with N even, point i sits at position (parity(i) ? M/2 : 0) + (i >> 1).
// (P,Q) is a vec2 array in that order; the (U,V) buffer holds U for all
// positions, then V for all positions (planar), so a gather of the other
// colour's U reads no V.  A colour pass then reads and writes its own colour's
// contiguous half and gathers the other half's neighbours with consecutive
// threads on consecutive elements.
__host__ __device__ __forceinline__ int point_parity(int64_t i, int dim, int64_t N)
{
    if (dim == 1) return (int)(i & 1);
    if (dim == 2) return (int)((i + i / N) & 1);
    return (int)((i + i / N + i / (N * N)) & 1);
}
__host__ __device__ __forceinline__ int64_t split_pos(int64_t i, int dim, int64_t N, int64_t half)
{
    return (point_parity(i, dim, N) ? half : 0) + (i >> 1);
}

// Largest point count the shared-memory resident kernel takes for state type T
// (whole (P,Q) and (U,V) arrays in one CTA's shared memory).
int64_t smem_resident_max_points(int elem_bytes);

// Sweep launchers (kgs_sweep.cu).  pq/uv hold the state as vec2 (P,Q) and (U,V)
// in natural order.  All launches go to `stream`; each returns the number of
// kernels it launched, or -1 if a launch failed (cudaGetLastError is set).
template <typename T>
int launch_pass(const Grid& g, int mode, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c,
                cudaStream_t stream);
template <typename T>
int launch_smem_run(const Grid& g, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c,
                    int64_t nsteps, cudaStream_t stream);

// One (BLACK_FUSED, red_mode) pair of colour passes in one cooperative launch
// (kgs_sweep.cu: wave_kernel): slabs of S axis-0 planes, chunks of `rows`
// rows, taken in a dependency-safe ticket order; red slab j waits for black
// slabs j-1, j, j+1.  wave_ctas: the launch's CTAs (all co-resident).
// wave_plan fills the parameters for a grid and that many CTAs (0), or
// returns -1 where the wave schedule does not apply (1D, N < 64, too few
// slabs for the lag).  sync: 2 + 2 ns unsigned words on the device (zeroed by the
// launcher on the stream); err: a word the kernel sets to 1 if a wait timed
// out (2 s; stall > 0 makes every wait need that many extra chunks, which
// tests the timeout).  launch_wave returns 1, or -1 if the launch failed.
struct WaveParams {
    int S = 0, ns = 0, rows = 0, chunks = 0, lag = 2, stall = 0;
};
int wave_ctas(int dim, int elem_bytes, int64_t M);
int wave_plan(int dim, int64_t N, int elem_bytes, int64_t want_S, int want_lag, int64_t want_chunk, int ctas,
              WaveParams& wp);
template <typename T>
int launch_wave(const Grid& g, int red_mode, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c,
                const WaveParams& wp, unsigned* sync, int* err, cudaStream_t s);

// Temporally blocked colour passes (kgs_tile.cu): passes g0 .. g0+P-1 of an
// nsteps-step run in one launch, reading (pq, uv) and writing (pq_out, uv_out).
struct TileParams {
    int64_t N = 0;        // set by the launcher
    int T1 = 32, T2 = 32; // tile extent along axis 1 and the last axis (2D: T2 only)
    int LX = 64;          // axis-0 planes per CTA
    int H = 4;            // halo width = largest pass count per launch
    int P = 4;            // passes in this launch (<= H)
    int threads = 256;
    int64_t g0 = 0;       // run index of the launch's first pass
    int64_t nsteps = 0;   // length of the run (its passes are 0 .. 2 nsteps)
};
int64_t tile_smem_bytes(int dim, int elem_bytes, const TileParams& tp);
template <typename T>
int launch_tile(const Grid& g, TileParams tp, const vec2_t<T>* pq, const vec2_t<T>* uv,
                vec2_t<T>* pq_out, vec2_t<T>* uv_out, const Coef<T>& c, cudaStream_t stream);

// Streamed planes (kgs_stream.cu): float32 3D step pairs, a step's black and
// red passes in one launch walking axis 0, planes staged by TMA tensor loads,
// on a private packed layout (per colour and plane, (N + 8) rows of N/2 + 4
// float4 (P, Q, U, V), with ghost copies of the periodic neighbours).
// stream_applies: whether a grid qualifies; stream_buffer_bytes: one packed
// copy of the state; stream_make_map: the TMA tensor map (a 64-byte aligned,
// 128-byte CUtensorMap at map_out) of a packed buffer, 0 or -1.
// launch_stream: one step pair (BLACK_FUSED, red_mode = RED_FUSED or
// RED_ADJ) reading the buffer of `map`, writing dst; err: the word a CTA sets
// to 2 if a bounded wait ran out (stall != 0 makes every CTA wait once on a
// barrier nothing completes).  chunk: 0 = each CTA a contiguous share of
// the (tile, plane) sequence; > 0 = items of `chunk` planes round-robin in
// chunk-major order (neighbouring tiles in step); prefetch: planes beyond
// the shared-memory loads also fetched into L2 (0: none).  launch_to_packed / launch_from_packed: the
// whole state between the colour-split layout and a packed buffer.  Each
// returns 1 (kernels launched) or -1 if a launch failed.
bool stream_applies(int dim, int64_t N, int precision);
size_t stream_buffer_bytes(int64_t N);
// The default chunk of planes per work item for a grid on `sms` SMs.
int stream_auto_chunk(int64_t N, int sms);
// steps: 1 for launch_stream's staged box, 2 for launch_stream2's.
int stream_make_map(void* buf, int64_t N, int steps, void* map_out);
int launch_stream(const void* map, void* dst, int64_t N, const Coef<float>& c, int red_mode, int* err, int stall,
                  int chunk, int prefetch, cudaStream_t s);
// Two steps per launch (temporal depth 2) on the same packed buffers:
// stream2_prepare writes the per-grid list of points beyond the tiles'
// columns (kStream2SideBytes at side_out; -1 if the grid's tiles do not fit
// the kernel's thread layout); launch_stream2 applies (BLACK_FUSED,
// RED_FUSED, BLACK_FUSED, red_mode), arguments otherwise as launch_stream's.
constexpr size_t kStream2SideBytes = 1024;
int stream2_auto_chunk(int64_t N, int sms);
int stream2_prepare(int64_t N, void* side_out);
int launch_stream2(const void* map, const void* side, void* dst, int64_t N, const Coef<float>& c, int red_mode,
                   int* err, int stall, int chunk, int prefetch, cudaStream_t s);
int launch_to_packed(const void* pq, const void* uv, void* out, int64_t N, cudaStream_t s);
int launch_from_packed(const void* in, void* pq, void* uv, int64_t N, cudaStream_t s);

// Update orders (kgs_order.cu).  order_schedule: level of every point of a
// permutation `order` of the N^dim grid (returns 0, -1 if order is not a
// permutation, -3 if host memory ran out).  order_lists: the points sorted by
// level (stable in order position), as packed coordinates (the last axis in
// the lowest bits, 63 / 31 / 21 bits per axis in 1 / 2 / 3 dimensions), and
// the level offsets (nlevels + 1).
// launch_level: one level's points, MODE RED_BASE (base half), RED_ADJ
// (adjoint half), PSI_HALF or UV_HALF (one variable's update alone, for
// per-variable orders), on the colour-split layout (split) or on natural vec2 order;
// returns 1, 0 for an empty level, -1 if the launch failed.
int order_schedule(int dim, int64_t N, const int64_t* order, int32_t* level, int64_t* nlevels);
int order_lists(int dim, int64_t N, const int64_t* order, std::vector<int64_t>& list,
                std::vector<int64_t>& offsets);
template <typename T>
int launch_level(int dim, int mode, vec2_t<T>* pq, vec2_t<T>* uv, const int64_t* list, int64_t count,
                 int64_t N, const Coef<T>& c, bool split, cudaStream_t s);
// launch_level_persistent: one whole step (base half up the levels, adjoint
// half down) in one cooperative launch of enough CTAs for the largest level
// (at most all co-resident CTAs), a bounded grid barrier after each level;
// offsets on the device (nlevels + 1); bar is zeroed on the stream first and
// bar->err is 1 afterwards if a barrier timed out.  extra > 0 makes every
// barrier wait for that many CTAs that do not exist (tests the timeout).
// Returns 1, or -1 if the launch failed.
struct OrderBarrier {
    unsigned count, gen;
    int err, pad;
};
template <typename T>
int launch_level_persistent(int dim, vec2_t<T>* pq, vec2_t<T>* uv, const int64_t* list,
                            const int64_t* offsets, int64_t nlevels, int64_t max_level, int64_t N,
                            const Coef<T>& c, OrderBarrier* bar, int extra, cudaStream_t s);

// The lexicographic order (and its reverse) in 2D as a doacross sweep
// (kgs_order.cu): one warp per strip of 32 rows, its lanes skewed by one
// column, each strip trailing the one before it; on natural vec2 order.
// lex_sweep_applies: whether the grid qualifies (dim 2, N a multiple of 32,
// N >= 64).  launch_lex_sweep: one half step (forward = increasing lex order)
// of MODE RED_BASE or RED_ADJ; sync: 2 + N/32 unsigned words on the device
// (zeroed by the launcher), err: a word set to 1 if a wait timed out (2 s;
// stall > 0 makes every wait need that many extra steps, which tests the
// timeout).  Returns 1, or -1 if the launch failed.
bool lex_sweep_applies(int dim, int64_t N);
template <typename T>
int launch_lex_sweep(bool forward, int mode, vec2_t<T>* pq, vec2_t<T>* uv, int64_t N, const Coef<T>& c,
                     unsigned* sync, int* err, int stall, cudaStream_t s);

// Layout conversion (kgs_layout.cu): one float64 field <-> one component of a
// vec2 array, natural order on the float64 side; dim > 0 puts the vec2 side in
// the colour-split layout of an N^dim grid, planar = the (U,V) buffer's planar
// form (component comp at comp M + position).  launch_split_convert: whole
// (P,Q) and (U,V) buffers between natural vec2 order and the colour-split
// layout (to_split: natural -> split).
template <typename T>
int launch_pack(int64_t M, vec2_t<T>* dst, int comp, const double* src, cudaStream_t stream,
                int dim = 0, int64_t N = 0, bool planar = false);
template <typename T>
int launch_unpack(int64_t M, double* dst, const vec2_t<T>* src, int comp, cudaStream_t stream,
                  int dim = 0, int64_t N = 0, bool planar = false);
template <typename T>
int launch_split_convert(const Grid& g, bool to_split, const vec2_t<T>* pq_in, const vec2_t<T>* uv_in,
                         vec2_t<T>* pq_out, vec2_t<T>* uv_out, cudaStream_t stream);

// Invariants (kgs_reduce.cu): E_h, its absolute-term scale, and the mass.
struct InvParams {
    double k1, k2;          // kappa1 / (2 h^2), kappa2 / (2 h^2)
    double abs_k1, abs_k2;  // their absolute values
    double mu2, gamma;      // mu^2, gamma
    double hd;              // h^dim
};
inline InvParams make_inv_params(int dim, double h, double kappa1, double kappa2, double mu, double gamma)
{
    InvParams p;
    p.k1 = kappa1 / (2.0 * h * h);
    p.k2 = kappa2 / (2.0 * h * h);
    p.abs_k1 = p.k1 < 0 ? -p.k1 : p.k1;
    p.abs_k2 = p.k2 < 0 ? -p.k2 : p.k2;
    p.mu2 = mu * mu;
    p.gamma = gamma;
    p.hd = 1.0;
    for (int a = 0; a < dim; ++a) p.hd *= h;
    return p;
}
int invariants_blocks(int dim, int64_t N);
template <typename T>
int launch_invariants(const Grid& g, const vec2_t<T>* pq, const vec2_t<T>* uv,
                      const InvParams& p, double* partials, int nblocks, double* out3,
                      cudaStream_t stream);

// Half-step coefficients of one problem (kgs_point.cuh), computed in FP64 on
// the host; the FP32 set is the FP64 one rounded.  One definition for the solo
// and batched paths, so both step an instance with the same constants.
inline Coef<double> host_coef64(int dim, int64_t N, double L, double kappa1, double kappa2,
                                double mu, double gamma, double tau)
{
    const double hh = L / (double)N;
    const double s = tau / 2.0, h2 = hh * hh, d = (double)dim;
    const double beta = s * kappa1 / (2.0 * h2);
    const double B = s * kappa2 / h2;
    const double A = d * B + s * mu * mu / 2.0;
    const double E = s * gamma;
    const double inv_det = 1.0 / (1.0 + A * s / 2.0);
    Coef<double> c;
    c.alpha = d * beta;
    c.g = s * gamma / 2.0;
    c.beta = beta;
    c.Bp = B * inv_det;
    c.Ep = E * inv_det;
    c.twoAp = 2.0 * A * inv_det;
    c.s = s;
    c.hs = s / 2.0;
    return c;
}

inline Coef<float> host_coef32(const Coef<double>& c)
{
    Coef<float> f;
    f.alpha = (float)c.alpha;
    f.g = (float)c.g;
    f.beta = (float)c.beta;
    f.Bp = (float)c.Bp;
    f.Ep = (float)c.Ep;
    f.twoAp = (float)c.twoAp;
    f.s = (float)c.s;
    f.hs = (float)c.hs;
    return f;
}

// Index checks of the KGS_DEBUG_BOUNDS build (libkgs_debug.so).  With the
// macro defined, a kernel checks its indices before an access and, where one
// is out of range, sets a bit of its file's device flag word and skips the
// access instead of trapping (the flags are read and cleared by
// kgs_debug_bounds, kgs_probe.h); without it the checks compile to nothing.
// Bits: 1 colour-pass indices, 2 streamed-plane shared-memory indices, 4
// streamed-plane stores, 8 batch indices.  KGS_BOUNDS_TU defines the flag
// word and kgs_in_bounds in a file, KGS_BOUNDS_READER(fn) its host reader.
#ifdef KGS_DEBUG_BOUNDS
#define KGS_BOUNDS_TU                                                                 \
    static __device__ unsigned kgs_bounds_flag_;                                     \
    static __device__ __forceinline__ bool kgs_in_bounds(bool ok, unsigned bit)      \
    {                                                                                 \
        if (!ok) atomicOr(&kgs_bounds_flag_, bit);                                    \
        return ok;                                                                    \
    }
#define KGS_BOUNDS_READER(fn)                                                         \
    unsigned fn()                                                                     \
    {                                                                                 \
        unsigned v = 0, z = 0;                                                        \
        if (cudaMemcpyFromSymbol(&v, kgs_bounds_flag_, sizeof v) != cudaSuccess) return ~0u; \
        if (cudaMemcpyToSymbol(kgs_bounds_flag_, &z, sizeof z) != cudaSuccess) return ~0u;   \
        return v;                                                                     \
    }
#else
#define KGS_BOUNDS_TU                                                                 \
    static __device__ __forceinline__ bool kgs_in_bounds(bool, unsigned) { return true; }
#define KGS_BOUNDS_READER(fn) \
    unsigned fn() { return 0u; }
#endif
unsigned bounds_flags_sweep();
unsigned bounds_flags_stream();
unsigned bounds_flags_batch();

// An NVTX range over a scope (kgs_step, kgs_invariants, the batch calls): a
// profiler attached to the process shows each call on its timeline; without
// one the push and pop return at once (NVTX v3, header only).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Record status and message as the calling thread's last error (what
// kgs_last_status / kgs_last_error return); returns status.
int report_error(int status, const char* msg);

}  // namespace kgs
