// kgs_api.cu -- the C ABI of libkgs (declared and documented in include/kgs.h).
//
// A handle owns its device state ((P,Q) and (U,V) as vec2 arrays in the state
// precision, in the colour-split layout of kgs_internal.h: each colour's points
// contiguous), a float64 staging buffer for layout conversion, and reduction
// scratch.  kgs_step issues the fused colour passes of a checkerboard DP-AVF2
// run (RED_BASE, (BLACK_FUSED, RED_FUSED) x (n-1), BLACK_FUSED, RED_ADJ; see
// kgs_point.cuh): small grids as one shared-memory resident launch, larger
// ones as one launch per pass, the repeated (BLACK_FUSED, RED_FUSED) pairs
// replayed from a captured CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/kgs.h"
#include "kgs_internal.h"

using namespace kgs;

namespace {

thread_local char g_last_error[512] = "";
thread_local int g_last_status = 0;

int fail(int status, const char* fmt, ...)
{
    g_last_status = status;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return status;
}

// Pairs of colour passes per captured graph.
constexpr int kGraphPairs = 32;

}  // namespace

struct kgs_solver {
    int dim = 0, precision = 64, device = 0;
    int64_t N = 0, M = 0;
    double L = 0, h = 0, kappa1 = 0, kappa2 = 0, mu = 0, gamma = 0, tau = 0;
    void* pqb[2] = {nullptr, nullptr};  // state buffers; [cur] holds the state
    void* uvb[2] = {nullptr, nullptr};  // ([1 - cur] is the tile kernel's output)
    int cur = 0;
    double* stage = nullptr;
    double* partials = nullptr;
    double* out_dev = nullptr;
    double* out_host = nullptr;
    int nblocks = 0;
    bool state_set = false;
    int sticky = 0;  // first CUDA error seen (cudaError_t), 0 if none
    int opt_kernel = 0, opt_graph = 1, opt_threads = 256;
    int opt_pdl = 1;  // programmatic dependent launch of the plain colour passes
    int64_t opt_slab = 0;  // planes per slab of the slab kernel (0: from the L2 size)
    TileParams tile{};
    bool tile_set = false;  // tile parameters chosen by the caller
    cudaStream_t last_stream = nullptr;
    int64_t launches = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_buf = -1;  // state buffer the graph was captured on
    int64_t graph_launches = 0;  // kernels per replay of the graph
    Coef<double> cd{};
    Coef<float> cf{};
    // update order other than the checkerboard (kgs_set_order): points sorted
    // by level on the device, level offsets on the host; empty = checkerboard
    int64_t* olist = nullptr;
    std::vector<int64_t> olevels;
    // a separate order for (U,V) (kgs_set_orders): its level list and offsets;
    // null = the same order as Psi (Algorithm 1's per-point procedure)
    int64_t* olist_uv = nullptr;
    std::vector<int64_t> olevels_uv;
    cudaGraphExec_t ograph = nullptr;  // one step of the order, captured
    int ograph_buf = -1;
    bool ograph_split = true;          // the layout the order graph was captured for
    int64_t* olevels_dev = nullptr;    // level offsets on the device (persistent launches)
    int64_t omax_level = 0;            // points in the largest level
    OrderBarrier* obar = nullptr;      // grid barrier of the persistent launches
    int opt_order_mode = 0;            // 0 auto, 1 levels on the split layout, 2 persistent, 3 levels on natural order, 4 lexicographic sweep
    int opt_stall = 0;                 // test hook: phantom CTAs every barrier waits for
    bool timed_out = false;            // a bounded device wait ran out: the state is lost
    // wave kernel (KGS_OPT_KERNEL 6): plan (0 not made, 1 usable, -1 not
    // applicable: plain passes), its counters and the timeout word (pinned,
    // mapped, so the host reads it without a copy)
    WaveParams wplan{};
    int wplan_state = 0;
    unsigned* wsync = nullptr;
    int* werr = nullptr;
    int opt_wave_lag = 0;
    int64_t opt_wave_chunk = 0;
    // the order is the lexicographic one (1) or its reverse (-1), 0 otherwise;
    // for grids lex_sweep_applies takes, the strip sweep's progress counters
    int olex = 0;
    unsigned* lsync = nullptr;
    // streamed-plane kernels (KGS_OPT_KERNEL 7, 8): two packed copies of the state
    // and their TMA tensor maps (CUtensorMap storage)
    void* sbuf[2] = {nullptr, nullptr};
    alignas(64) unsigned char smap[2][128] = {};
    // two steps per launch (KGS_OPT_KERNEL 8): the staged box's tensor maps
    // and the grid's side list (sside_ok: stream2_prepare succeeded)
    alignas(64) unsigned char smap2[2][128] = {};
    alignas(16) unsigned char sside[kStream2SideBytes] = {};
    bool sside_ok = false;
    int opt_stream_chunk = 0;  // KGS_OPT_STREAM_CHUNK
    // device bytes this handle may allocate (KGS_DEVICE_BUDGET at creation; 0 =
    // no limit) and the bytes it holds
    size_t budget = 0, dev_bytes = 0;
    int opt_stream_prefetch = -1;  // KGS_OPT_STREAM_PREFETCH (-1: default)
};

namespace {

// Makes h's device current for the duration of a call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int cuda_fail(kgs_solver* h, cudaError_t e, const char* what)
{
    if (h && !h->sticky) h->sticky = (int)e;
    return fail(KGS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int check_handle(kgs_solver* h)
{
    if (!h) return fail(KGS_ERR_ARG, "NULL handle");
    if (h->werr && *(volatile int*)h->werr) h->timed_out = true;
    if (h->timed_out)
        return fail(KGS_ERR_TIMEOUT, "handle is in error state after a device wait timed out");
    if (h->sticky)
        return fail(KGS_ERR_CUDA, "handle is in error state after: %s",
                    cudaGetErrorString((cudaError_t)h->sticky));
    return KGS_OK;
}

bool is_finite_(double x) { return std::isfinite(x); }

// A device allocation of the handle, counted against its budget: with the
// environment variable KGS_DEVICE_BUDGET set (bytes, read by kgs_create) an
// allocation that would take the handle past it fails on the host as if the
// device were out of memory -- the way to make an allocation fail on purpose
// (tests of the KGS_ERR_OOM paths) without exhausting a shared device.
cudaError_t hmalloc(kgs_solver* h, void** p, size_t bytes)
{
    if (h->budget && h->dev_bytes + bytes > h->budget) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) h->dev_bytes += bytes;
    return e;
}

void hfree(kgs_solver* h, void* p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    h->dev_bytes -= bytes < h->dev_bytes ? bytes : h->dev_bytes;
}

void compute_coef(kgs_solver* h)
{
    h->cd = host_coef64(h->dim, h->N, h->L, h->kappa1, h->kappa2, h->mu, h->gamma, h->tau);
    h->cf = host_coef32(h->cd);
}

void drop_graph(kgs_solver* h)
{
    // a replay of either graph may still be queued: let it finish first
    if (h->graph || h->ograph) cudaDeviceSynchronize();
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (h->ograph) {
        cudaGraphExecDestroy(h->ograph);
        h->ograph = nullptr;
    }
}

int kernel_choice(const kgs_solver* h);

Grid grid_of(const kgs_solver* h)
{
    Grid g{h->dim, h->N, h->M};
    g.threads = h->opt_threads;
    g.persistent = kernel_choice(h) == 4;
    g.split = true;  // a handle's state is in the colour-split layout
    return g;
}

enum KernelChoice {
    K_PASS = 1, K_SMEM = 2, K_TILE = 3, K_PERSIST = 4, K_SLAB = 5, K_WAVE = 6, K_STREAM = 7, K_STREAM2 = 8
};

// Default tile shape per dimension and precision (measured on B300; the batch
// autotuner can override it per handle).
TileParams default_tile(int dim, int precision)
{
    TileParams t;
    if (dim == 2) {
        t.T1 = 1; t.T2 = 256; t.LX = 64; t.H = t.P = 8; t.threads = 512;
    } else if (precision == 32) {
        t.T1 = 32; t.T2 = 32; t.LX = 64; t.H = t.P = 3; t.threads = 512;
    } else {
        t.T1 = 16; t.T2 = 16; t.LX = 64; t.H = t.P = 2; t.threads = 512;
    }
    return t;
}

int kernel_choice(const kgs_solver* h)
{
    const int64_t cap = smem_resident_max_points(h->precision == 64 ? 8 : 4);
    if (h->opt_kernel >= K_PASS && h->opt_kernel <= K_STREAM2) return h->opt_kernel;
    if (h->M <= cap) return K_SMEM;
    // Float32 3D grids the streamed-plane kernels take, from N = 128: two steps
    // per launch (measured, point-updates/s against one launch per pass: 512^3
    // 1.46e11 / 1.09e11, 256^3 1.22e11 / 1.01e11, 128^3 6.6e10 / 5.2e10; at
    // 64^3 the grid's 3 tiles leave most SMs idle: 9.4e9 / 2.3e10).
    if (stream_applies(h->dim, h->N, h->precision) && h->N >= 128) return K_STREAM2;
    // Otherwise, measured on B300 (3D 512^3 / 2D 2048^2): one launch per pass
    // beats the temporally blocked tiles in both precisions (FP32: 8.6e10 vs
    // 6.2e10 / 9.8e10 vs 3.4e10 point-updates/s; FP64: 1.0e10 vs 6.1e9), so
    // the tile kernel is chosen only on request (KGS_OPT_KERNEL = 3).
    return K_PASS;
}

int ensure_tile_buffers(kgs_solver* h)
{
    if (h->pqb[1]) return 0;
    const size_t elem = h->precision == 64 ? sizeof(double2) : sizeof(float2);
    const size_t bytes = (size_t)h->M * elem;
    cudaError_t e = hmalloc(h, &h->pqb[1], bytes);
    if (e == cudaSuccess) e = hmalloc(h, &h->uvb[1], bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hfree(h, h->pqb[1], bytes);
        h->pqb[1] = nullptr;
        h->uvb[1] = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? KGS_ERR_OOM : KGS_ERR_CUDA,
                    "second state buffer (%zu bytes): %s", 2 * bytes,
                    cudaGetErrorString(e));
    }
    return 0;
}

int ensure_err_word(kgs_solver* h);

// The streamed-plane kernel's packed buffers and tensor maps (first use).
int ensure_stream(kgs_solver* h)
{
    if (h->sbuf[1]) return KGS_OK;
    if (ensure_err_word(h)) return KGS_ERR_OOM;
    const size_t bytes = stream_buffer_bytes(h->N);
    cudaError_t e = hmalloc(h, &h->sbuf[0], bytes);
    if (e == cudaSuccess) e = hmalloc(h, &h->sbuf[1], bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hfree(h, h->sbuf[0], bytes);
        h->sbuf[0] = h->sbuf[1] = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? KGS_ERR_OOM : KGS_ERR_CUDA,
                    "streamed-plane buffers (2 x %zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    for (int b = 0; b < 2; ++b) {
        if (stream_make_map(h->sbuf[b], h->N, 1, h->smap[b]) || stream_make_map(h->sbuf[b], h->N, 2, h->smap2[b])) {
            hfree(h, h->sbuf[0], bytes);
            hfree(h, h->sbuf[1], bytes);
            h->sbuf[0] = h->sbuf[1] = nullptr;
            return fail(KGS_ERR_CUDA, "TMA tensor map of the streamed-plane buffers");
        }
    }
    h->sside_ok = stream2_prepare(h->N, h->sside) == 0;
    return KGS_OK;
}

template <typename T>
int pass(kgs_solver* h, int mode, cudaStream_t s)
{
    const Coef<T>* c;
    if constexpr (sizeof(T) == 8) c = &h->cd;
    else c = &h->cf;
    int n = launch_pass<T>(grid_of(h), mode, (vec2_t<T>*)h->pqb[h->cur], (vec2_t<T>*)h->uvb[h->cur],
                           *c, s);
    if (n < 0) return -1;
    h->launches += n;
    return 0;
}

// Planes per slab: the caller's choice, else about a quarter of L2 per slab.
int64_t slab_planes(const kgs_solver* h)
{
    if (h->opt_slab > 0) return h->opt_slab < h->N ? h->opt_slab : h->N;
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device) != cudaSuccess || l2 <= 0)
        l2 = 126 << 20;
    const int64_t plane = h->M / h->N * 2 * (h->precision == 64 ? 16 : 8);
    int64_t p = (int64_t)(l2 / 4) / plane;
    if (p < 2) p = 2;
    return p < h->N ? p : h->N;
}

// The word a bounded device wait sets when it times out: pinned host memory
// mapped into the device, so the host reads it without a copy.
int ensure_err_word(kgs_solver* h)
{
    if (h->werr) return KGS_OK;
    cudaError_t e = cudaHostAlloc(&h->werr, sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->werr = nullptr;
        return fail(KGS_ERR_OOM, "pinned error word: %s", cudaGetErrorString(e));
    }
    *(volatile int*)h->werr = 0;
    return KGS_OK;
}

// The wave kernel's plan and buffers; returns 1 if it applies to the grid, 0
// if not (the plain passes run instead), or a negative status.
int ensure_wave(kgs_solver* h)
{
    if (h->wplan_state) return h->wplan_state > 0;
    WaveParams wp;
    const int elem = h->precision == 64 ? 8 : 4;
    if (wave_plan(h->dim, h->N, elem, h->opt_slab, h->opt_wave_lag, h->opt_wave_chunk, wave_ctas(h->dim, elem, h->M),
                  wp)) {
        h->wplan_state = -1;
        return 0;
    }
    cudaFree(h->wsync);
    h->wsync = nullptr;
    cudaError_t e = cudaMalloc(&h->wsync, (size_t)(2 + 2 * wp.ns) * sizeof(unsigned));
    if (e == cudaSuccess && ensure_err_word(h)) return KGS_ERR_OOM;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? KGS_ERR_OOM : KGS_ERR_CUDA, "wave kernel buffers: %s",
                    cudaGetErrorString(e));
    }
    h->wplan = wp;
    h->wplan_state = 1;
    return 1;
}

// A wave launch whose wait timed out leaves the state undefined; read after
// a synchronisation of the handle's work.
int wave_status(kgs_solver* h)
{
    if (h->werr && *(volatile int*)h->werr) {
        h->timed_out = true;
        return fail(KGS_ERR_TIMEOUT, "a dependency wait of the wave kernel timed out");
    }
    return KGS_OK;
}

// One (BLACK_FUSED, red) pair of colour passes, red = RED_FUSED or RED_ADJ.
// With the slab kernel the black pass runs slab by slab along axis 0 and the
// red pass of slab s - 1 follows the black pass of slab s: the red pass of a
// plane needs the black planes on both sides updated, and the black pass of a
// plane needs the red planes on both sides not yet updated, so red plane 0
// (whose lower neighbour is black plane N - 1, by periodicity) goes last.
template <typename T>
int pass_pair(kgs_solver* h, int red, cudaStream_t s)
{
    const Coef<T>* c;
    if constexpr (sizeof(T) == 8) c = &h->cd;
    else c = &h->cf;
    vec2_t<T>* pq = (vec2_t<T>*)h->pqb[h->cur];
    vec2_t<T>* uv = (vec2_t<T>*)h->uvb[h->cur];
    Grid g = grid_of(h);
    if (kernel_choice(h) == K_WAVE) {
        const int w = ensure_wave(h);
        if (w < 0) return -1;
        if (w > 0) {
            WaveParams wp = h->wplan;
            wp.stall = h->opt_stall;
            if (launch_wave<T>(g, red, pq, uv, *c, wp, h->wsync, h->werr, s) < 0) return -1;
            h->launches += 1;
            return 0;
        }
    }
    if (kernel_choice(h) != K_SLAB || h->dim < 2) {
        g.pdl = g.pdl_wait = h->opt_pdl != 0;
        if (launch_pass<T>(g, BLACK_FUSED, pq, uv, *c, s) < 0 || launch_pass<T>(g, red, pq, uv, *c, s) < 0)
            return -1;
        h->launches += 2;
        return 0;
    }
    const int64_t S = slab_planes(h), N = h->N;
    const int64_t ns = (N + S - 1) / S;
    // the pair's first two launches (black slabs 0 and 1) wait for everything
    // before them; the others are programmatic dependent launches (see
    // pass_kernel): from the third on, every red launch waits for the black
    // one just before it, and every black launch starts only after the red
    // one before it has passed that wait, so each red slab finds its three
    // black slabs complete
    int index = 0;
    auto run = [&](int mode, int64_t p0, int64_t p1) -> int {
        if (p1 <= p0) return 0;
        g.plane0 = p0;
        g.planes = p1 - p0;
        g.pdl = index++ >= 2;
        if (launch_pass<T>(g, mode, pq, uv, *c, s) < 0) return -1;
        h->launches += 1;
        return 0;
    };
    auto end = [&](int64_t k) { return (k + 1) * S < N ? (k + 1) * S : N; };
    if (run(BLACK_FUSED, 0, end(0))) return -1;
    for (int64_t k = 1; k < ns; ++k) {
        if (run(BLACK_FUSED, k * S, end(k))) return -1;
        if (run(red, k == 1 ? 1 : (k - 1) * S, end(k - 1))) return -1;
    }
    if (run(red, ns == 1 ? 1 : (ns - 1) * S, N)) return -1;
    return run(red, 0, 1);
}

template <typename T>
int ensure_graph(kgs_solver* h)
{
    if (h->graph && h->graph_buf == h->cur) return 0;
    drop_graph(h);
    // allocations are not allowed while a stream is being captured
    if (kernel_choice(h) == K_WAVE && ensure_wave(h) < 0) return KGS_ERR_CUDA;
    if (!h->capture_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreate");
    }
    cudaError_t e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
    const Coef<T>* c;
    if constexpr (sizeof(T) == 8) c = &h->cd;
    else c = &h->cf;
    const int64_t l0 = h->launches;
    int bad = 0;
    for (int k = 0; k < kGraphPairs && !bad; ++k) bad = pass_pair<T>(h, RED_FUSED, h->capture_stream);
    h->graph_launches = h->launches - l0;
    h->launches = l0;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->capture_stream, &graph);
    if (bad && e == cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(h, cudaErrorLaunchFailure, "colour pass capture");
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    h->graph_buf = h->cur;
    return 0;
}

// One DP-AVF2 step in the handle's order: the base half over the levels in
// increasing order, the adjoint half in decreasing order.
// One sweep over an order's levels (upward = the order's direction) in mode m.
template <typename T>
int order_sweep(kgs_solver* h, const int64_t* list, const std::vector<int64_t>& levels, bool upward, int m,
                bool split, cudaStream_t s)
{
    const Coef<T>* c;
    if constexpr (sizeof(T) == 8) c = &h->cd;
    else c = &h->cf;
    vec2_t<T>* pq = (vec2_t<T>*)h->pqb[h->cur];
    vec2_t<T>* uv = (vec2_t<T>*)h->uvb[h->cur];
    const int64_t nl = (int64_t)levels.size() - 1;
    for (int64_t k = 0; k < nl; ++k) {
        const int64_t l = upward ? k : nl - 1 - k;
        const int64_t o = levels[(size_t)l], n = levels[(size_t)l + 1] - o;
        const int r = launch_level<T>(h->dim, m, pq, uv, list + o, n, h->N, *c, split, s);
        if (r < 0) return -1;
        h->launches += r;
    }
    return 0;
}

// One step in the handle's order(s): the base half up the levels, the adjoint
// half down; with a separate (U,V) order, each half is two sweeps (base: Psi
// in its order, then (U,V) in its order; adjoint: (U,V), then Psi, both
// reversed) -- with one order the same arithmetic as the per-point form.
template <typename T>
int order_step(kgs_solver* h, bool split, cudaStream_t s)
{
    if (!h->olist_uv)
        return order_sweep<T>(h, h->olist, h->olevels, true, RED_BASE, split, s) ||
                       order_sweep<T>(h, h->olist, h->olevels, false, RED_ADJ, split, s)
                   ? -1
                   : 0;
    if (order_sweep<T>(h, h->olist, h->olevels, true, PSI_HALF, split, s) ||
        order_sweep<T>(h, h->olist_uv, h->olevels_uv, true, UV_HALF, split, s) ||
        order_sweep<T>(h, h->olist_uv, h->olevels_uv, false, UV_HALF, split, s) ||
        order_sweep<T>(h, h->olist, h->olevels, false, PSI_HALF, split, s))
        return -1;
    return 0;
}

template <typename T>
int step_in_order_persistent(kgs_solver* h, int64_t nsteps, cudaStream_t s)
{
    const Coef<T>* c;
    if constexpr (sizeof(T) == 8) c = &h->cd;
    else c = &h->cf;
    const int64_t nl = (int64_t)h->olevels.size() - 1;
    cudaError_t e = cudaMemsetAsync(h->obar, 0, sizeof(OrderBarrier), s);
    if (e != cudaSuccess) return cuda_fail(h, e, "barrier reset");
    for (int64_t k = 0; k < nsteps; ++k) {
        // count and generation restart each launch; the error flag is kept
        e = cudaMemsetAsync(h->obar, 0, 2 * sizeof(unsigned), s);
        if (e != cudaSuccess) return cuda_fail(h, e, "barrier reset");
        if (launch_level_persistent<T>(h->dim, (vec2_t<T>*)h->pqb[h->cur], (vec2_t<T>*)h->uvb[h->cur],
                                       h->olist, h->olevels_dev, nl, h->omax_level, h->N, *c, h->obar,
                                       h->opt_stall, s) < 0)
            return cuda_fail(h, cudaGetLastError(), "persistent order launch");
        h->launches += 1;
    }
    int err = 0;
    e = cudaMemcpyAsync(&err, &h->obar->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "barrier status");
    if (err) {
        h->timed_out = true;
        return fail(KGS_ERR_TIMEOUT, "a level barrier of the persistent order launch timed out");
    }
    return KGS_OK;
}

// Levels on natural vec2 order: convert the state into the other buffer pair
// (to_natural) or back into the colour-split layout, and make that pair current.
template <typename T>
int order_convert(kgs_solver* h, bool to_natural, cudaStream_t s)
{
    if (to_natural) {
        const int st = ensure_tile_buffers(h);
        if (st) return st;
    }
    const int o = h->cur ^ 1;
    if (launch_split_convert<T>(grid_of(h), !to_natural, (const vec2_t<T>*)h->pqb[h->cur],
                                (const vec2_t<T>*)h->uvb[h->cur], (vec2_t<T>*)h->pqb[o], (vec2_t<T>*)h->uvb[o],
                                s) < 0)
        return cuda_fail(h, cudaGetLastError(), "layout conversion");
    h->launches += 1;
    h->cur = o;
    return KGS_OK;
}

template <typename T>
int step_in_order_levels(kgs_solver* h, int64_t nsteps, bool split, cudaStream_t s);

// The lexicographic order (or its reverse) as a doacross sweep of row strips:
// per step the base half in the order's direction, the adjoint half in the
// other.
template <typename T>
int step_in_order_lex(kgs_solver* h, int64_t nsteps, cudaStream_t s)
{
    const Coef<T>* c;
    if constexpr (sizeof(T) == 8) c = &h->cd;
    else c = &h->cf;
    vec2_t<T>* pq = (vec2_t<T>*)h->pqb[h->cur];
    vec2_t<T>* uv = (vec2_t<T>*)h->uvb[h->cur];
    const bool fwd = h->olex > 0;
    for (int64_t k = 0; k < nsteps; ++k) {
        if (launch_lex_sweep<T>(fwd, RED_BASE, pq, uv, h->N, *c, h->lsync, h->werr, h->opt_stall, s) < 0 ||
            launch_lex_sweep<T>(!fwd, RED_ADJ, pq, uv, h->N, *c, h->lsync, h->werr, h->opt_stall, s) < 0)
            return cuda_fail(h, cudaGetLastError(), "lexicographic sweep launch");
        h->launches += 2;
    }
    return KGS_OK;
}

template <typename T>
int step_in_order(kgs_solver* h, int64_t nsteps, cudaStream_t s)
{
    if (h->opt_order_mode == 2 && !h->olist_uv) return step_in_order_persistent<T>(h, nsteps, s);
    // natural order suits the level schedules better: a level's points (an
    // anti-diagonal of the lexicographic order, say) find their neighbours
    // along the last axis in the cache sectors of their own values
    bool natural = h->opt_order_mode == 3 || h->opt_order_mode == 4;
    if (h->opt_order_mode == 0) {
        // without room for the copy, fall back to the levels on the split
        // layout, leaving the caller's last-error record as it was
        const int saved = g_last_status;
        char msg[sizeof g_last_error];
        memcpy(msg, g_last_error, sizeof msg);
        natural = ensure_tile_buffers(h) == 0;
        if (!natural) {
            g_last_status = saved;
            memcpy(g_last_error, msg, sizeof msg);
        }
    }
    const bool lex = natural && h->olex != 0 && h->lsync && !h->olist_uv &&
                     (h->opt_order_mode == 0 || h->opt_order_mode == 4);
    if (natural) {
        int st = order_convert<T>(h, true, s);
        if (st) return st;
        st = lex ? step_in_order_lex<T>(h, nsteps, s) : step_in_order_levels<T>(h, nsteps, false, s);
        const int st2 = order_convert<T>(h, false, s);
        return st ? st : st2;
    }
    return step_in_order_levels<T>(h, nsteps, true, s);
}

template <typename T>
int step_in_order_levels(kgs_solver* h, int64_t nsteps, bool split, cudaStream_t s)
{
    if (h->opt_graph && nsteps >= 2) {
        if (!(h->ograph && h->ograph_buf == h->cur && h->ograph_split == split)) {
            if (h->ograph) {
                cudaGraphExecDestroy(h->ograph);
                h->ograph = nullptr;
            }
            if (!h->capture_stream) {
                cudaError_t e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
                if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreate");
            }
            cudaError_t e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
            const int64_t l0 = h->launches;
            const int r = order_step<T>(h, split, h->capture_stream);
            h->launches = l0;
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(h->capture_stream, &graph);
            if (r < 0 && e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(h, e == cudaSuccess ? cudaErrorUnknown : e, "order step capture");
            }
            e = cudaGraphInstantiate(&h->ograph, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                h->ograph = nullptr;
                return cuda_fail(h, e, "cudaGraphInstantiate");
            }
            h->ograph_buf = h->cur;
            h->ograph_split = split;
        }
        int64_t per = 0;
        for (size_t l = 0; l + 1 < h->olevels.size(); ++l) per += h->olevels[l + 1] > h->olevels[l];
        for (size_t l = 0; l + 1 < h->olevels_uv.size(); ++l) per += h->olevels_uv[l + 1] > h->olevels_uv[l];
        for (int64_t k = 0; k < nsteps; ++k) {
            cudaError_t e = cudaGraphLaunch(h->ograph, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
            h->launches += 2 * per;
        }
        return KGS_OK;
    }
    for (int64_t k = 0; k < nsteps; ++k)
        if (order_step<T>(h, split, s)) return cuda_fail(h, cudaGetLastError(), "order level launch");
    return KGS_OK;
}

template <typename T>
int step_impl(kgs_solver* h, int64_t nsteps, cudaStream_t s)
{
    if (!h->olevels.empty()) return step_in_order<T>(h, nsteps, s);
    const Coef<T>* c;
    if constexpr (sizeof(T) == 8) c = &h->cd;
    else c = &h->cf;
    const int kc = kernel_choice(h);
    if (kc == K_SMEM) {
        int n = launch_smem_run<T>(grid_of(h), (vec2_t<T>*)h->pqb[h->cur], (vec2_t<T>*)h->uvb[h->cur],
                                   *c, nsteps, s);
        if (n < 0) return cuda_fail(h, cudaGetLastError(), "shared-memory run launch");
        h->launches += n;
        return KGS_OK;
    }
    if (kc == K_TILE) {
        int st = ensure_tile_buffers(h);
        if (st) return st;
        TileParams tp = h->tile_set ? h->tile : default_tile(h->dim, h->precision);
        const int64_t passes = 2 * nsteps + 1;
        const int per = tp.H;
        // the tile kernel works on natural order: convert into the other buffer
        // pair, run, convert back (the state ends in buffer pair cur)
        {
            const int o = h->cur ^ 1;
            if (launch_split_convert<T>(grid_of(h), false, (const vec2_t<T>*)h->pqb[h->cur],
                                        (const vec2_t<T>*)h->uvb[h->cur], (vec2_t<T>*)h->pqb[o],
                                        (vec2_t<T>*)h->uvb[o], s) < 0)
                return cuda_fail(h, cudaGetLastError(), "layout conversion");
            h->launches += 1;
            h->cur = o;
        }
        for (int64_t g0 = 0; g0 < passes; g0 += per) {
            tp.g0 = g0;
            tp.nsteps = nsteps;
            tp.P = (int)((passes - g0) < per ? (passes - g0) : per);
            const int o = h->cur ^ 1;
            int n = launch_tile<T>(grid_of(h), tp, (const vec2_t<T>*)h->pqb[h->cur],
                                   (const vec2_t<T>*)h->uvb[h->cur], (vec2_t<T>*)h->pqb[o],
                                   (vec2_t<T>*)h->uvb[o], *c, s);
            if (n < 0) {
                cudaError_t e = cudaGetLastError();
                if (e == cudaSuccess)
                    return fail(KGS_ERR_ARG, "tile parameters not usable for this grid");
                return cuda_fail(h, e, "tile kernel launch");
            }
            h->launches += n;
            h->cur = o;
        }
        {
            const int o = h->cur ^ 1;
            if (launch_split_convert<T>(grid_of(h), true, (const vec2_t<T>*)h->pqb[h->cur],
                                        (const vec2_t<T>*)h->uvb[h->cur], (vec2_t<T>*)h->pqb[o],
                                        (vec2_t<T>*)h->uvb[o], s) < 0)
                return cuda_fail(h, cudaGetLastError(), "layout conversion");
            h->launches += 1;
            h->cur = o;
        }
        return KGS_OK;
    }
    if constexpr (sizeof(T) == 4) {
        if ((kc == K_STREAM || kc == K_STREAM2) && stream_applies(h->dim, h->N, h->precision)) {
            // R_base on the handle's layout, then the steps streamed on the packed
            // copies -- two per launch (KGS_OPT_KERNEL 8) or one, the last with
            // the adjoint red half -- and back
            int st = ensure_stream(h);
            if (st) return st;
            if (pass<T>(h, RED_BASE, s)) return cuda_fail(h, cudaGetLastError(), "colour pass launch");
            if (launch_to_packed(h->pqb[h->cur], h->uvb[h->cur], h->sbuf[0], h->N, s) < 0)
                return cuda_fail(h, cudaGetLastError(), "layout conversion");
            int sms = 148;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
            const bool two = kc == K_STREAM2 && h->sside_ok;
            // chunk planes: the caller's, or the grid's default
            const int chunk1 = h->opt_stream_chunk == 0 ? stream_auto_chunk(h->N, sms)
                                                        : (h->opt_stream_chunk < 0 ? 0 : h->opt_stream_chunk);
            const int chunk2 = h->opt_stream_chunk == 0 ? stream2_auto_chunk(h->N, sms)
                                                        : (h->opt_stream_chunk < 0 ? 0 : h->opt_stream_chunk);
            // L2 prefetch distance: the caller's, or 2 planes (one step per launch at 512^3: 1 / 2 / 4
            // planes 0.733 / 0.732 / 0.730 of HBM; two steps: 2 and 6 planes alike, 1.714 / 1.715 ms)
            const int pf = h->opt_stream_prefetch < 0 ? 2 : h->opt_stream_prefetch;
            int cs = 0;
            int64_t nl = 0;
            for (int64_t k = 0; k < nsteps; ++nl) {
                const int take = two && nsteps - k >= 2 ? 2 : 1;
                const int mode = k + take == nsteps ? RED_ADJ : RED_FUSED;
                const int r = take == 2 ? launch_stream2(h->smap2[cs], h->sside, h->sbuf[cs ^ 1], h->N, h->cf, mode,
                                                         h->werr, h->opt_stall, chunk2, pf, s)
                                        : launch_stream(h->smap[cs], h->sbuf[cs ^ 1], h->N, h->cf, mode, h->werr,
                                                        h->opt_stall, chunk1, pf, s);
                if (r < 0) return cuda_fail(h, cudaGetLastError(), "streamed-plane launch");
                cs ^= 1;
                k += take;
            }
            if (launch_from_packed(h->sbuf[cs], h->pqb[h->cur], h->uvb[h->cur], h->N, s) < 0)
                return cuda_fail(h, cudaGetLastError(), "layout conversion");
            h->launches += nl + 2;  // (the R_base pass counted itself)
            return KGS_OK;
        }
    }
    if (pass<T>(h, RED_BASE, s)) return cuda_fail(h, cudaGetLastError(), "colour pass launch");
    int64_t pairs = nsteps - 1;
    if (h->opt_graph && pairs >= kGraphPairs) {
        if (ensure_graph<T>(h)) return KGS_ERR_CUDA;
        while (pairs >= kGraphPairs) {
            cudaError_t e = cudaGraphLaunch(h->graph, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
            h->launches += h->graph_launches;
            pairs -= kGraphPairs;
        }
    }
    for (; pairs > 0; --pairs) {
        if (pass_pair<T>(h, RED_FUSED, s)) return cuda_fail(h, cudaGetLastError(), "colour pass launch");
    }
    if (pass_pair<T>(h, RED_ADJ, s)) return cuda_fail(h, cudaGetLastError(), "colour pass launch");
    return KGS_OK;
}

void free_all(kgs_solver* h)
{
    cudaDeviceSynchronize();  // no queued work may still use what is freed below
    drop_graph(h);
    cudaFree(h->olist);
    cudaFree(h->olist_uv);
    cudaFree(h->olevels_dev);
    cudaFree(h->obar);
    cudaFree(h->wsync);
    cudaFree(h->lsync);
    h->lsync = nullptr;
    if (h->werr) cudaFreeHost(h->werr);
    h->wsync = nullptr;
    h->werr = nullptr;
    h->olist = nullptr;
    h->olevels_dev = nullptr;
    h->obar = nullptr;
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->pqb[b]);
        cudaFree(h->uvb[b]);
    }
    cudaFree(h->sbuf[0]);
    cudaFree(h->sbuf[1]);
    cudaFree(h->stage);
    cudaFree(h->partials);
    cudaFree(h->out_dev);
    if (h->out_host) cudaFreeHost(h->out_host);
}

}  // namespace

int kgs::report_error(int status, const char* msg) { return fail(status, "%s", msg); }

extern "C" {

kgs_handle kgs_create_ex(int dim, int64_t N, double L, double kappa1, double kappa2, double mu,
                         double gamma, double tau, int precision, int device)
{
    g_last_error[0] = '\0';
    g_last_status = KGS_OK;
    if (dim < 1 || dim > 3) { fail(KGS_ERR_ARG, "dim must be 1, 2 or 3 (got %d)", dim); return nullptr; }
    if (N < 4 || (N & 1)) {
        fail(KGS_ERR_ODD_N, "N must be even and >= 4 (got %lld)", (long long)N);
        return nullptr;
    }
    // 1D: one row; 2D: rows are launch-grid y indices (<= 65535); 3D: 4096^3 points
    if (N > (int64_t)1 << 30 || (dim == 2 && N > 65534) || (dim == 3 && N > 4096)) {
        fail(KGS_ERR_RANGE, "N^d too large (dim %d, N %lld)", dim, (long long)N);
        return nullptr;
    }
    if (!is_finite_(L) || L <= 0) { fail(KGS_ERR_ARG, "L must be finite and > 0"); return nullptr; }
    if (!is_finite_(kappa1) || !is_finite_(kappa2) || !is_finite_(mu) || !is_finite_(gamma)) {
        fail(KGS_ERR_ARG, "kappa1, kappa2, mu, gamma must be finite");
        return nullptr;
    }
    if (!is_finite_(tau) || tau == 0.0) { fail(KGS_ERR_ARG, "tau must be finite and nonzero"); return nullptr; }
    if (precision != KGS_FP64 && precision != KGS_FP32) {
        fail(KGS_ERR_ARG, "precision must be KGS_FP64 or KGS_FP32 (got %d)", precision);
        return nullptr;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        fail(KGS_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
        return nullptr;
    }
    if (device < 0) {
        if (cudaGetDevice(&device) != cudaSuccess) { fail(KGS_ERR_CUDA, "cudaGetDevice failed"); return nullptr; }
    }
    if (device >= ndev) { fail(KGS_ERR_ARG, "device %d out of range (%d devices)", device, ndev); return nullptr; }
    DeviceGuard guard(device);
    if (!guard.ok) { fail(KGS_ERR_CUDA, "cudaSetDevice(%d) failed", device); return nullptr; }

    kgs_solver* h = new (std::nothrow) kgs_solver();
    if (!h) { fail(KGS_ERR_OOM, "host allocation failed"); return nullptr; }
    h->dim = dim;
    h->N = N;
    h->M = 1;
    for (int a = 0; a < dim; ++a) h->M *= N;
    h->L = L;
    h->h = L / (double)N;
    h->kappa1 = kappa1;
    h->kappa2 = kappa2;
    h->mu = mu;
    h->gamma = gamma;
    h->tau = tau;
    h->precision = precision;
    h->device = device;
    compute_coef(h);
    const size_t elem = precision == 64 ? sizeof(double2) : sizeof(float2);
    const size_t state_bytes = (size_t)h->M * elem;
    h->nblocks = invariants_blocks(h->dim, h->N);
    if (const char* b = std::getenv("KGS_DEVICE_BUDGET")) h->budget = (size_t)std::strtoull(b, nullptr, 10);
    cudaError_t ea = hmalloc(h, &h->pqb[0], state_bytes);
    if (ea == cudaSuccess) ea = hmalloc(h, &h->uvb[0], state_bytes);
    if (ea == cudaSuccess) ea = hmalloc(h, (void**)&h->stage, (size_t)h->M * sizeof(double));
    if (ea == cudaSuccess) ea = hmalloc(h, (void**)&h->partials, (size_t)h->nblocks * 3 * sizeof(double));
    if (ea == cudaSuccess) ea = hmalloc(h, (void**)&h->out_dev, 3 * sizeof(double));
    if (ea == cudaSuccess) ea = cudaMallocHost(&h->out_host, 3 * sizeof(double));
    if (ea != cudaSuccess) {
        cudaGetLastError();
        int status = (ea == cudaErrorMemoryAllocation) ? KGS_ERR_OOM : KGS_ERR_CUDA;
        fail(status, "device allocation of %zu state bytes failed: %s", 2 * state_bytes,
             cudaGetErrorString(ea));
        free_all(h);
        delete h;
        return nullptr;
    }
    return h;
}

kgs_handle kgs_create(int dim, int64_t N, double L, double kappa1, double kappa2, double mu,
                      double gamma, double tau)
{
    return kgs_create_ex(dim, N, L, kappa1, kappa2, mu, gamma, tau, KGS_FP64, -1);
}

int kgs_set_state(kgs_handle h, const double* P, const double* Q, const double* U, const double* V,
                  int where, void* stream)
{
    int st = check_handle(h);
    if (st) return st;
    if (!P || !Q || !U || !V) return fail(KGS_ERR_ARG, "NULL state pointer");
    if (where != KGS_HOST && where != KGS_DEVICE && where != KGS_HOST_ASYNC)
        return fail(KGS_ERR_ARG, "where must be KGS_HOST, KGS_DEVICE or KGS_HOST_ASYNC");
    DeviceGuard guard(h->device);
    if (!guard.ok) return cuda_fail(h, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const double* src[4] = {P, Q, U, V};
    const bool host = where != KGS_DEVICE;
    for (int f = 0; f < 4; ++f) {
        const double* d = src[f];
        if (host) {
            cudaError_t e = cudaMemcpyAsync(h->stage, src[f], (size_t)h->M * sizeof(double),
                                            cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "state upload");
            d = h->stage;
        }
        void* dst = (f < 2) ? h->pqb[h->cur] : h->uvb[h->cur];
        int n = (h->precision == 64)
                    ? launch_pack<double>(h->M, (double2*)dst, f & 1, d, s, h->dim, h->N, f >= 2)
                    : launch_pack<float>(h->M, (float2*)dst, f & 1, d, s, h->dim, h->N, f >= 2);
        if (n < 0) return cuda_fail(h, cudaGetLastError(), "pack launch");
        h->launches += n;
    }
    if (where == KGS_HOST) {  // (KGS_HOST_ASYNC: the caller waits for the stream)
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    }
    h->state_set = true;
    h->last_stream = s;
    return KGS_OK;
}

int kgs_get_state(kgs_handle h, double* P, double* Q, double* U, double* V, int where, void* stream)
{
    int st = check_handle(h);
    if (st) return st;
    if (!h->state_set) return fail(KGS_ERR_STATE, "no state set");
    if (!P || !Q || !U || !V) return fail(KGS_ERR_ARG, "NULL state pointer");
    if (where != KGS_HOST && where != KGS_DEVICE && where != KGS_HOST_ASYNC)
        return fail(KGS_ERR_ARG, "where must be KGS_HOST, KGS_DEVICE or KGS_HOST_ASYNC");
    DeviceGuard guard(h->device);
    if (!guard.ok) return cuda_fail(h, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    double* dst[4] = {P, Q, U, V};
    const bool host = where != KGS_DEVICE;
    for (int f = 0; f < 4; ++f) {
        double* d = host ? h->stage : dst[f];
        const void* src = (f < 2) ? h->pqb[h->cur] : h->uvb[h->cur];
        int n = (h->precision == 64)
                    ? launch_unpack<double>(h->M, d, (const double2*)src, f & 1, s, h->dim, h->N, f >= 2)
                    : launch_unpack<float>(h->M, d, (const float2*)src, f & 1, s, h->dim, h->N, f >= 2);
        if (n < 0) return cuda_fail(h, cudaGetLastError(), "unpack launch");
        h->launches += n;
        if (host) {
            cudaError_t e = cudaMemcpyAsync(dst[f], h->stage, (size_t)h->M * sizeof(double),
                                            cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "state download");
        }
    }
    if (where == KGS_HOST) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
        return wave_status(h);
    }
    return KGS_OK;
}

int kgs_step(kgs_handle h, int64_t nsteps, void* stream)
{
    NvtxRange range("kgs_step");
    int st = check_handle(h);
    if (st) return st;
    if (nsteps < 0) return fail(KGS_ERR_ARG, "nsteps must be >= 0");
    if (!h->state_set) return fail(KGS_ERR_STATE, "no state set");
    h->last_stream = (cudaStream_t)stream;
    if (nsteps == 0) return KGS_OK;
    DeviceGuard guard(h->device);
    if (!guard.ok) return cuda_fail(h, cudaGetLastError(), "cudaSetDevice");
    return h->precision == 64 ? step_impl<double>(h, nsteps, (cudaStream_t)stream)
                              : step_impl<float>(h, nsteps, (cudaStream_t)stream);
}

int kgs_order_schedule(int dim, int64_t N, const int64_t* order, int32_t* level, int64_t* nlevels)
{
    g_last_status = KGS_OK;
    if (dim < 1 || dim > 3) return fail(KGS_ERR_ARG, "dim must be 1, 2 or 3 (got %d)", dim);
    if (N < 4 || (N & 1)) return fail(KGS_ERR_ODD_N, "N must be even and >= 4 (got %lld)", (long long)N);
    if ((dim == 3 && N > 4096) || (dim == 2 && N > 65534) || N > ((int64_t)1 << 30))
        return fail(KGS_ERR_RANGE, "N^d too large");
    if (!order || !level || !nlevels) return fail(KGS_ERR_ARG, "NULL argument");
    const int st = order_schedule(dim, N, order, level, nlevels);
    if (st == -3) return fail(KGS_ERR_OOM, "host memory for the order schedule");
    if (st) return fail(KGS_ERR_ARG, "order is not a permutation of 0 .. N^d - 1");
    return KGS_OK;
}

int kgs_set_order(kgs_handle h, const int64_t* order)
{
    int st = check_handle(h);
    if (st) return st;
    DeviceGuard guard(h->device);
    if (!guard.ok) return cuda_fail(h, cudaGetLastError(), "cudaSetDevice");
    // the previous order's list may still be read by queued work
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
    drop_graph(h);
    // validate before changing anything: a rejected order leaves the handle's order(s) as they were
    std::vector<int64_t> list, off;
    if (order) {
        st = order_lists(h->dim, h->N, order, list, off);
        if (st == -3) return fail(KGS_ERR_OOM, "host memory for the order schedule");
        if (st) return fail(KGS_ERR_ARG, "order is not a permutation of 0 .. N^d - 1");
    }
    h->olex = 0;
    cudaFree(h->olist_uv);
    h->olist_uv = nullptr;
    h->olevels_uv.clear();
    if (!order) {
        cudaFree(h->olist);
        cudaFree(h->olevels_dev);
        h->olist = nullptr;
        h->olevels_dev = nullptr;
        h->olevels.clear();
        return KGS_OK;
    }
    if (!h->olist) {
        e = cudaMalloc(&h->olist, (size_t)h->M * sizeof(int64_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->olist = nullptr;
            return fail(KGS_ERR_OOM, "device memory for the order (%lld points)", (long long)h->M);
        }
    }
    e = cudaMemcpy(h->olist, list.data(), (size_t)h->M * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "order upload");
    cudaFree(h->olevels_dev);
    h->olevels_dev = nullptr;
    e = cudaMalloc(&h->olevels_dev, off.size() * sizeof(int64_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(h->olevels_dev, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !h->obar) e = cudaMalloc(&h->obar, sizeof(OrderBarrier));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KGS_ERR_OOM, "device memory for the order's level offsets");
    }
    h->omax_level = 0;
    for (size_t l = 0; l + 1 < off.size(); ++l) h->omax_level = std::max(h->omax_level, off[l + 1] - off[l]);
    h->olevels.swap(off);
    // the lexicographic order or its reverse: the tile sweep applies
    h->olex = 0;
    bool fwd = true, bwd = true;
    for (int64_t i = 0; i < h->M && (fwd || bwd); ++i) {
        fwd = fwd && order[i] == i;
        bwd = bwd && order[i] == h->M - 1 - i;
    }
    if ((fwd || bwd) && lex_sweep_applies(h->dim, h->N)) {
        if (!h->lsync) {
            e = cudaMalloc(&h->lsync, (size_t)(2 + h->N / 32) * sizeof(unsigned));
            if (e != cudaSuccess) {
                cudaGetLastError();
                h->lsync = nullptr;
                return fail(KGS_ERR_OOM, "device memory for the lexicographic sweep");
            }
        }
        if ((st = ensure_err_word(h))) return st;
        h->olex = fwd ? 1 : -1;
    }
    return KGS_OK;
}

int kgs_set_orders(kgs_handle h, const int64_t* order_psi, const int64_t* order_uv)
{
    int st = check_handle(h);
    if (st) return st;
    if (!order_psi || !order_uv) return fail(KGS_ERR_ARG, "both orders are required (kgs_set_order resets)");
    // validate the (U,V) order before changing anything
    std::vector<int64_t> list, off;
    st = order_lists(h->dim, h->N, order_uv, list, off);
    if (st == -3) return fail(KGS_ERR_OOM, "host memory for the order schedule");
    if (st) return fail(KGS_ERR_ARG, "order_uv is not a permutation of 0 .. N^d - 1");
    if ((st = kgs_set_order(h, order_psi))) return st;  // clears any earlier (U,V) order
    if (std::equal(order_psi, order_psi + h->M, order_uv)) return KGS_OK;  // one common order
    DeviceGuard guard(h->device);
    if (!guard.ok) return cuda_fail(h, cudaGetLastError(), "cudaSetDevice");
    cudaError_t e = cudaMalloc(&h->olist_uv, (size_t)h->M * sizeof(int64_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->olist_uv = nullptr;
        return fail(KGS_ERR_OOM, "device memory for the (U,V) order (%lld points)", (long long)h->M);
    }
    e = cudaMemcpy(h->olist_uv, list.data(), (size_t)h->M * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "order upload");
    h->olevels_uv.swap(off);
    h->olex = 0;  // the lexicographic sweep runs one common order only
    return KGS_OK;
}

int kgs_order_levels(kgs_handle h, int64_t* nlevels)
{
    int st = check_handle(h);
    if (st) return st;
    if (!nlevels) return fail(KGS_ERR_ARG, "NULL output");
    *nlevels = h->olevels.empty() ? 2 : (int64_t)h->olevels.size() - 1 + (int64_t)h->olevels_uv.size() -
                                            (h->olevels_uv.empty() ? 0 : 1);
    return KGS_OK;
}

int kgs_invariants(kgs_handle h, double* out3, void* stream)
{
    NvtxRange range("kgs_invariants");
    int st = check_handle(h);
    if (st) return st;
    if (!out3) return fail(KGS_ERR_ARG, "NULL output");
    if (!h->state_set) return fail(KGS_ERR_STATE, "no state set");
    DeviceGuard guard(h->device);
    if (!guard.ok) return cuda_fail(h, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const InvParams p = make_inv_params(h->dim, h->h, h->kappa1, h->kappa2, h->mu, h->gamma);
    int n = (h->precision == 64)
                ? launch_invariants<double>(grid_of(h), (const double2*)h->pqb[h->cur],
                                            (const double2*)h->uvb[h->cur], p, h->partials,
                                            h->nblocks, h->out_dev, s)
                : launch_invariants<float>(grid_of(h), (const float2*)h->pqb[h->cur],
                                           (const float2*)h->uvb[h->cur], p, h->partials,
                                           h->nblocks, h->out_dev, s);
    if (n < 0) return cuda_fail(h, cudaGetLastError(), "invariants launch");
    h->launches += n;
    cudaError_t e = cudaMemcpyAsync(h->out_host, h->out_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "invariants readback");
    if ((st = wave_status(h))) return st;
    for (int k = 0; k < 3; ++k) out3[k] = h->out_host[k];
    return KGS_OK;
}

int kgs_energy(kgs_handle h, double* E)
{
    if (!E) return fail(KGS_ERR_ARG, "NULL output");
    double out[3];
    int st = kgs_invariants(h, out, h ? (void*)h->last_stream : nullptr);
    if (st == KGS_OK) *E = out[0];
    return st;
}

int kgs_mass(kgs_handle h, double* M)
{
    if (!M) return fail(KGS_ERR_ARG, "NULL output");
    double out[3];
    int st = kgs_invariants(h, out, h ? (void*)h->last_stream : nullptr);
    if (st == KGS_OK) *M = out[2];
    return st;
}

int kgs_set_tau(kgs_handle h, double tau)
{
    int st = check_handle(h);
    if (st) return st;
    if (!is_finite_(tau) || tau == 0.0) return fail(KGS_ERR_ARG, "tau must be finite and nonzero");
    h->tau = tau;
    compute_coef(h);
    drop_graph(h);
    return KGS_OK;
}

int kgs_set_option(kgs_handle h, int option, int64_t value)
{
    int st = check_handle(h);
    if (st) return st;
    switch (option) {
    case KGS_OPT_KERNEL:
        if (value < 0 || value > 8) return fail(KGS_ERR_ARG, "KGS_OPT_KERNEL takes 0 to 8");
        if (value == 5 && h->dim < 2) return fail(KGS_ERR_ARG, "the slab kernel needs dim 2 or 3");
        if (value == 6 && h->dim < 2) return fail(KGS_ERR_ARG, "the wave kernel needs dim 2 or 3");
        if (value == 2 && h->M > smem_resident_max_points(h->precision == 64 ? 8 : 4))
            return fail(KGS_ERR_RANGE, "grid too large for the shared-memory resident kernel");
        if (value == 3 && h->dim < 2)
            return fail(KGS_ERR_ARG, "the tile kernel needs dim 2 or 3");
        h->opt_kernel = (int)value;
        drop_graph(h);
        return KGS_OK;
    case KGS_OPT_TILE_T1:
    case KGS_OPT_TILE_T2:
    case KGS_OPT_TILE_LX:
    case KGS_OPT_TILE_PASSES:
    case KGS_OPT_TILE_THREADS: {
        if (!h->tile_set) {
            h->tile = default_tile(h->dim, h->precision);
            h->tile_set = true;
        }
        TileParams t = h->tile;
        const int v = (int)value;
        if (value < 1 || value > 4096) return fail(KGS_ERR_ARG, "tile option out of range");
        if (option == KGS_OPT_TILE_T1) t.T1 = v;
        else if (option == KGS_OPT_TILE_T2) t.T2 = v;
        else if (option == KGS_OPT_TILE_LX) t.LX = v;
        else if (option == KGS_OPT_TILE_PASSES) t.H = t.P = v;
        else {
            if (v != 64 && v != 128 && v != 256 && v != 512 && v != 1024)
                return fail(KGS_ERR_ARG, "tile threads take 64, 128, 256, 512 or 1024");
            t.threads = v;
        }
        if (t.H > 8 || t.T2 < 2 || (t.T2 & 1) || (h->dim == 3 && t.T1 < 2))
            return fail(KGS_ERR_ARG, "tile shape out of range");
        if (tile_smem_bytes(h->dim, h->precision == 64 ? 8 : 4, t) > 227 * 1024)
            return fail(KGS_ERR_RANGE, "tile shape needs more than 227 KB of shared memory");
        h->tile = t;
        return KGS_OK;
    }
    case KGS_OPT_GRAPH:
        if (value < 0 || value > 1) return fail(KGS_ERR_ARG, "KGS_OPT_GRAPH takes 0 or 1");
        h->opt_graph = (int)value;
        return KGS_OK;
    case KGS_OPT_ORDER_MODE:
        if (value < 0 || value > 4) return fail(KGS_ERR_ARG, "KGS_OPT_ORDER_MODE takes 0 to 4");
        h->opt_order_mode = (int)value;
        return KGS_OK;
    case KGS_OPT_TEST_BARRIER_STALL:
        if (value < 0 || value > 1024) return fail(KGS_ERR_ARG, "KGS_OPT_TEST_BARRIER_STALL takes 0 to 1024");
        h->opt_stall = (int)value;
        return KGS_OK;
    case KGS_OPT_SLAB_PLANES:
        if (value < 0 || value > h->N) return fail(KGS_ERR_ARG, "KGS_OPT_SLAB_PLANES takes 0 to N");
        h->opt_slab = value;
        h->wplan_state = 0;
        drop_graph(h);
        return KGS_OK;
    case KGS_OPT_WAVE_CHUNK:
        if (value < 0 || value > ((int64_t)1 << 24)) return fail(KGS_ERR_ARG, "KGS_OPT_WAVE_CHUNK takes 0 to 2^24");
        h->opt_wave_chunk = value;
        h->wplan_state = 0;
        drop_graph(h);
        return KGS_OK;
    case KGS_OPT_WAVE_LAG:
        if (value < 0 || value > 64) return fail(KGS_ERR_ARG, "KGS_OPT_WAVE_LAG takes 0 to 64");
        h->opt_wave_lag = (int)value;
        h->wplan_state = 0;
        drop_graph(h);
        return KGS_OK;
    case KGS_OPT_THREADS:
        if (value != 128 && value != 256 && value != 512)
            return fail(KGS_ERR_ARG, "KGS_OPT_THREADS takes 128, 256 or 512");
        h->opt_threads = (int)value;
        drop_graph(h);
        return KGS_OK;
    case KGS_OPT_STREAM_CHUNK:
        if (value < -1 || value > 65536) return fail(KGS_ERR_ARG, "KGS_OPT_STREAM_CHUNK takes -1 to 65536");
        h->opt_stream_chunk = (int)value;
        return KGS_OK;
    case KGS_OPT_STREAM_PREFETCH:
        if (value < 0 || value > 16) return fail(KGS_ERR_ARG, "KGS_OPT_STREAM_PREFETCH takes 0 to 16");
        h->opt_stream_prefetch = (int)value;
        return KGS_OK;
    case KGS_OPT_PDL:
        if (value < 0 || value > 1) return fail(KGS_ERR_ARG, "KGS_OPT_PDL takes 0 or 1");
        h->opt_pdl = (int)value;
        drop_graph(h);
        return KGS_OK;
    case KGS_OPT_PPT:
        if (value != 1) return fail(KGS_ERR_ARG, "KGS_OPT_PPT takes 1 (more points per thread "
                                                   "measured no faster on B300)");
        return KGS_OK;
    default:
        return fail(KGS_ERR_ARG, "unknown option %d", option);
    }
}

int64_t kgs_launch_count(kgs_handle h) { return h ? h->launches : -1; }

void kgs_destroy(kgs_handle h)
{
    if (!h) return;
    {
        DeviceGuard guard(h->device);
        free_all(h);
    }
    delete h;
}

const char* kgs_strerror(int status)
{
    switch (status) {
    case KGS_OK: return "ok";
    case KGS_ERR_ARG: return "invalid argument";
    case KGS_ERR_ODD_N: return "N must be even and >= 4";
    case KGS_ERR_OOM: return "device out of memory";
    case KGS_ERR_CUDA: return "CUDA error";
    case KGS_ERR_STATE: return "no state set";
    case KGS_ERR_TIMEOUT: return "device wait timed out";
    case KGS_ERR_RANGE: return "size out of supported range";
    default: return "unknown status";
    }
}

const char* kgs_last_error(void) { return g_last_error; }

int kgs_last_status(void) { return g_last_status; }

}  // extern "C"
