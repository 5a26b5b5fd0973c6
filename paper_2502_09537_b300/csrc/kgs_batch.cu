// kgs_batch.cu -- many independent KGS instances of different sizes,
// dimensions and precisions stepped together (declared in include/kgs.h,
// kgs_batch_*).
//
// Storage: one device arena per batch, of a capacity fixed at creation (the
// HBM budget), holding every instance's (P,Q) vec2 array and (U,V) buffer in
// the colour-split layout of a handle's state (kgs_internal.h); instances
// are placed first-fit and their space is returned on removal, so a caller can
// admit new instances as others finish.
//
// Stepping: a DP-AVF2 step of every instance is two colour passes (kgs_point.cuh:
// RED_BASE, (BLACK_FUSED, RED_FUSED) x (n-1), BLACK_FUSED, RED_ADJ).  Pass g of
// every instance is applied by a persistent grid of CTAs walking a work list of
// 256-point chunks of the instances' points of that colour, one launch per
// precision, dimension and pass mode that occurs at pass g (each kernel is
// specialised on them); a chunk's instance is read from a table built with the
// list.  Each instance i may run its own number of steps n_i; pass g of its
// run is applied while g <= 2 n_i and skipped after.  The
// launches of a kgs_batch_step_each call are captured once into a CUDA graph
// and replayed while the instance set and step counts stay the same.  Each
// (precision, dimension) list's launch sequence runs on its own stream forked
// from the caller's and joined at the end: the lists hold disjoint instances,
// so their passes overlap (FP64 passes bound by the FP64 pipe beside FP32
// passes bound by DRAM, and one list's pass filling another's tail).  Every
// point update is the code of a solo run with the same neighbour order, so
// each instance's state is bitwise that of stepping it alone.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <new>
#include <vector>

#include "../../include/kgs.h"
#include "kgs_internal.h"

using namespace kgs;

namespace kgs {
KGS_BOUNDS_TU
KGS_BOUNDS_READER(bounds_flags_batch)
}  // namespace kgs

namespace {

constexpr int kChunk = 256;  // colour points per work item (= CTA size)

template <typename T> struct BatchInst {
    vec2_t<T>* pq;
    vec2_t<T>* uv;
    int dim, N;
    int64_t half;         // points of one colour
    int64_t first_chunk;  // prefix of chunks over the instances of this list
    int64_t nsteps;       // steps of the current call (0: idle)
    Coef<T> coef;
};

__device__ __forceinline__ int batch_mode(int64_t g, int64_t n)
{
    if (g == 0) return RED_BASE;
    if (g == 2 * n) return RED_ADJ;
    return (g & 1) ? BLACK_FUSED : RED_FUSED;
}

// Linear index and neighbours of the t-th point of a colour (0-based index sum
// parity `parity`) -- the same point order and neighbour order as the solo
// pass kernel; rows along the last axis, N/2 points of each colour per row.
template <int D, typename I>
__device__ __forceinline__ I batch_point(I t, int N, int parity, I nb[2 * D])
{
    const I hN = (I)(N >> 1);
    const I row = t / hN;
    const int kk = (int)(t - row * hN);
    int i0 = 0, i1 = 0, rp = 0;
    if (D == 2) {
        i0 = (int)row;
        rp = i0 & 1;
    } else if (D == 3) {
        i0 = (int)(row / N);
        i1 = (int)(row - (I)i0 * N);
        rp = (i0 + i1) & 1;
    }
    const int k = 2 * kk + ((parity - rp) & 1);
    const I n = N;
    const I i = row * n + k;
    const I km = (k == 0) ? i + (n - 1) : i - 1;
    const I kp = (k == N - 1) ? i - (n - 1) : i + 1;
    if (D == 1) {
        nb[0] = km;
        nb[1] = kp;
    } else if (D == 2) {
        nb[0] = (i0 == 0) ? i + (n - 1) * n : i - n;
        nb[1] = (i0 == N - 1) ? i - (n - 1) * n : i + n;
        nb[2] = km;
        nb[3] = kp;
    } else {
        const I n2 = n * n;
        nb[0] = (i0 == 0) ? i + (n - 1) * n2 : i - n2;
        nb[1] = (i0 == N - 1) ? i - (n - 1) * n2 : i + n2;
        nb[2] = (i1 == 0) ? i + (n - 1) * n : i - n;
        nb[3] = (i1 == N - 1) ? i - (n - 1) * n : i + n;
        nb[4] = km;
        nb[5] = kp;
    }
    return i;
}

// An instance's state is in the colour-split layout of a handle's
// (kgs_internal.h): this colour's half from pq + own, the neighbours in the
// other half, U and V planar in the (U,V) buffer.
// COHERENT: read the other colour's values with loads that bypass L1 (.cg),
// for the persistent kernel, where other CTAs wrote them during the same
// launch (L1 is not coherent across SMs); otherwise the read-only path.
template <typename T, int D, int MODE, typename I, bool COHERENT = false>
__device__ __forceinline__ void batch_update(const BatchInst<T>& in, I t, int parity)
{
    I nb[2 * D];
    const I i = batch_point<D, I>(t, in.N, parity, nb);
    const I half = (I)in.half;
    const I own = (parity ? half : 0) + (i >> 1);
    const I oth = parity ? 0 : half;
    T* u = reinterpret_cast<T*>(in.uv);
    {
        bool ok = own >= 0 && own < 2 * half;
#pragma unroll
        for (int m = 0; m < 2 * D; ++m) ok = ok && oth + (nb[m] >> 1) >= 0 && oth + (nb[m] >> 1) < 2 * half;
        if (!kgs::kgs_in_bounds(ok, 8u)) return;
    }
    T p[2 * D], q[2 * D], w[2 * D];
#pragma unroll
    for (int m = 0; m < 2 * D; ++m) {
        const I k = oth + (nb[m] >> 1);
        const vec2_t<T> b = COHERENT ? __ldcg(&in.pq[k]) : __ldg(&in.pq[k]);
        p[m] = b.x;
        q[m] = b.y;
        w[m] = COHERENT ? __ldcg(&u[k]) : __ldg(&u[k]);
    }
    vec2_t<T> a = COHERENT ? __ldcg(&in.pq[own]) : in.pq[own];
    T U = COHERENT ? __ldcg(&u[own]) : u[own], V = COHERENT ? __ldcg(&u[2 * half + own]) : u[2 * half + own];
    // FP64 V additions here: under the batch kernels' 64-register cap the
    // integer form spills (measured 1.3% slower on the batch workload, 2D)
    update_point<T, D, MODE, false, false>(in.coef, nsum_scaled(p, in.coef.beta), nsum_scaled(q, in.coef.beta),
                                    nsum_scaled(w, in.coef.Bp), a.x, a.y, U, V);
    in.pq[own] = a;
    u[own] = U;
    u[2 * half + own] = V;
}

// Pass g (colour: red for even g) of the instances of one list (one precision
// and dimension) whose mode at pass g is MODE; chunk_inst gives each chunk's
// instance, so a chunk's lookup is one load shared by the CTA.
// I: index type, int32_t when every instance of the list has fewer than 2^31 points.
template <typename T, int D, int MODE, typename I>
// Occupancy: FP64 passes are bound by the FP64 pipe and keep 4 CTAs per SM (64
// registers); FP32 passes are bound by memory latency and take 8 (32
// registers, no spills: measured 9.52e10 -> 1.05e11 on the batch workload).
__global__ void __launch_bounds__(kChunk, sizeof(T) == 4 ? 8 : 4) batch_pass_kernel(const BatchInst<T>* __restrict__ insts,
                                                            const int32_t* __restrict__ chunk_inst,
                                                            int64_t total_chunks, int64_t g)
{
    const int red = red_parity(D);
    const int parity = (g & 1) ? (red ^ 1) : red;
    for (int64_t ch = blockIdx.x; ch < total_chunks; ch += gridDim.x) {
        const BatchInst<T>& in = insts[__ldg(&chunk_inst[ch])];
        const int64_t n = in.nsteps;
        if (g > 2 * n || batch_mode(g, n) != MODE) continue;  // the same for the whole CTA
        const int64_t t = (ch - in.first_chunk) * kChunk + threadIdx.x;
        if (t >= in.half) continue;
        batch_update<T, D, MODE, I>(in, (I)t, parity);
    }
}

// ---- one persistent launch for a whole kgs_batch_step call ----------------
// Every pass g = 0 .. 2 nmax of every list (both precisions, every dimension)
// in one cooperative launch: per pass the CTAs walk the lists' chunks as one
// index space (a chunk's list is the same for the whole CTA), the mode of each
// instance at pass g decides its update, and a grid barrier ends the pass.
// The barrier is bounded (kPersistWaitNs of %globaltimer): a CTA that waits
// longer sets the error word and every CTA leaves.  Each chunk is updated by
// the same CTA every pass; neighbour values written by other CTAs in the pass
// before are read with L1-bypassing loads.
struct PersistLists {
    const void* inst[6];          // BatchInst<double> for k < 3, BatchInst<float> after; k % 3 = dim - 1
    const int32_t* chunk_inst[6];
    int64_t chunks[6];
    int64_t passes;               // 2 nmax + 1
};
struct BatchBarrier {
    unsigned count, gen;
    int err, pad;
};
constexpr uint64_t kPersistWaitNs = 2000000000ull;

__device__ __forceinline__ uint64_t batch_clock_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool batch_grid_sync(BatchBarrier* bar, unsigned expected, unsigned& gen)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's updates before its arrival
        if (atomicAdd(&bar->count, 1u) == expected - 1u) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const uint64_t t0 = batch_clock_ns();
            while (atomicAdd(&bar->gen, 0u) == gen) {
                if (atomicAdd(&bar->err, 0) != 0) break;
                if (batch_clock_ns() - t0 > kPersistWaitNs) {
                    atomicExch(&bar->err, 1);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();  // the other CTAs' updates before this CTA's next reads
    }
    ++gen;
    __syncthreads();
    return *(volatile int*)&bar->err == 0;
}

template <typename T, int D>
__device__ __forceinline__ void persist_chunk(const PersistLists& pl, int k, int64_t lc, int64_t g)
{
    const BatchInst<T>* insts = reinterpret_cast<const BatchInst<T>*>(pl.inst[k]);
    const BatchInst<T>& in = insts[__ldg(&pl.chunk_inst[k][lc])];
    const int64_t n = in.nsteps;
    if (g > 2 * n) return;
    const int64_t t = (lc - in.first_chunk) * kChunk + threadIdx.x;
    if (t >= in.half) return;
    const int red = red_parity(D);
    const int parity = (g & 1) ? (red ^ 1) : red;
    switch (batch_mode(g, n)) {
    case RED_BASE: batch_update<T, D, RED_BASE, int32_t, true>(in, (int32_t)t, parity); break;
    case BLACK_FUSED: batch_update<T, D, BLACK_FUSED, int32_t, true>(in, (int32_t)t, parity); break;
    case RED_FUSED: batch_update<T, D, RED_FUSED, int32_t, true>(in, (int32_t)t, parity); break;
    default: batch_update<T, D, RED_ADJ, int32_t, true>(in, (int32_t)t, parity); break;
    }
}

// expected = gridDim.x normally; the test hook sets it higher (the barrier
// then waits for CTAs that do not exist and times out).
__global__ void __launch_bounds__(kChunk, 4) batch_persistent_kernel(PersistLists pl, BatchBarrier* bar,
                                                                     unsigned expected, int* err)
{
    int64_t prefix[7];
    prefix[0] = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) prefix[k + 1] = prefix[k] + pl.chunks[k];
    unsigned gen = 0;
    for (int64_t g = 0; g < pl.passes; ++g) {
        for (int64_t ch = blockIdx.x; ch < prefix[6]; ch += gridDim.x) {
            int k = 0;
            while (ch >= prefix[k + 1]) ++k;
            const int64_t lc = ch - prefix[k];
            switch (k) {
            case 0: persist_chunk<double, 1>(pl, k, lc, g); break;
            case 1: persist_chunk<double, 2>(pl, k, lc, g); break;
            case 2: persist_chunk<double, 3>(pl, k, lc, g); break;
            case 3: persist_chunk<float, 1>(pl, k, lc, g); break;
            case 4: persist_chunk<float, 2>(pl, k, lc, g); break;
            default: persist_chunk<float, 3>(pl, k, lc, g); break;
            }
        }
        if (!batch_grid_sync(bar, expected, gen)) {
            if (threadIdx.x == 0) *(volatile int*)err = 1;
            return;
        }
    }
}

thread_local char g_batch_err[256];

int bfail(int status, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_batch_err, sizeof g_batch_err, fmt, ap);
    va_end(ap);
    return report_error(status, g_batch_err);
}

struct HostInst {
    bool live = false;
    int dim = 0, precision = 64;
    int64_t N = 0, M = 0;
    double L = 0, kappa1 = 0, kappa2 = 0, mu = 0, gamma = 0, tau = 0;
    size_t off = 0, bytes = 0;  // arena range: (P,Q) array then (U,V) array
    bool state_set = false;
};

}  // namespace

struct kgs_batch {
    int device = 0;
    char* arena = nullptr;
    size_t capacity = 0;
    std::map<size_t, size_t> free_ranges;  // offset -> length
    std::vector<HostInst> inst;
    // device work lists per precision (0: FP64, 1: FP32) and dimension: the
    // instance descriptors and the instance of every chunk
    struct DevList {
        void* inst = nullptr;
        int cap = 0;
        int32_t* chunk_inst = nullptr;
        int64_t chunk_cap = 0;
    } lists[2][3];
    int64_t graph_launches = 0;  // kernels per replay of the graph
    // stepping
    int ctas_per_sm = 8;
    int ctas_list[2][3] = {{0, 0, 0}, {0, 0, 0}};  // per (precision, dimension); 0 = ctas_per_sm
    int use_graph = 1;
    // one persistent cooperative launch per call (KGS_BATCH_OPT_PERSISTENT),
    // its grid barrier, the error word its bounded waits set (pinned, mapped)
    // and the test hook's phantom CTAs
    int persistent = 0;
    int stall = 0;
    BatchBarrier* pbar = nullptr;
    int* perr = nullptr;
    bool timed_out = false;
    bool persist_nograph = false;  // this driver refused to capture the cooperative launch
    cudaGraphExec_t graph = nullptr;
    std::vector<int64_t> graph_key;  // step counts the graph was captured for
    cudaEvent_t graph_ev = nullptr;  // recorded after each launch of the graph
    // graphs replaced while a launch of theirs may still run: destroyed once
    // the event recorded after that launch has completed
    std::vector<std::pair<cudaGraphExec_t, cudaEvent_t>> retired;
    cudaStream_t capture_stream = nullptr;
    cudaStream_t side[6] = {};              // streams of the lists after the first
    cudaEvent_t fork = nullptr, join[6] = {};
    int64_t launches = 0;
    int sticky = 0;
    double* scratch = nullptr;  // invariants partials
    double* out_dev = nullptr;
    double* out_host = nullptr;
    int scratch_blocks = 0;
};

namespace {

struct BatchDevGuard {
    int prev = -1;
    bool ok = true;
    explicit BatchDevGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~BatchDevGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int bcuda(kgs_batch* b, cudaError_t e, const char* what)
{
    if (b && !b->sticky) b->sticky = (int)e;
    return bfail(KGS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int bcheck(kgs_batch* b)
{
    if (!b) return bfail(KGS_ERR_ARG, "NULL batch handle");
    if (b->perr && *(volatile int*)b->perr) b->timed_out = true;
    if (b->timed_out)
        return bfail(KGS_ERR_TIMEOUT, "batch is in error state after a device wait timed out");
    if (b->sticky)
        return bfail(KGS_ERR_CUDA, "batch is in error state after: %s",
                     cudaGetErrorString((cudaError_t)b->sticky));
    return KGS_OK;
}

// Destroy the retired graphs whose last launch has completed (all of them,
// waiting if need be, when wait is set).
void reap_graphs(kgs_batch* b, bool wait)
{
    size_t keep = 0;
    for (auto& r : b->retired) {
        if (wait) cudaEventSynchronize(r.second);
        if (cudaEventQuery(r.second) == cudaSuccess) {
            cudaGraphExecDestroy(r.first);
            cudaEventDestroy(r.second);
        } else {
            b->retired[keep++] = r;
        }
    }
    b->retired.resize(keep);
    cudaGetLastError();  // a pending query is not an error
}

void drop_batch_graph(kgs_batch* b)
{
    if (b->graph) {
        if (b->graph_ev) {
            b->retired.emplace_back(b->graph, b->graph_ev);
            b->graph_ev = nullptr;
        } else {
            cudaGraphExecDestroy(b->graph);  // never launched
        }
    }
    b->graph = nullptr;
    b->graph_key.clear();
    reap_graphs(b, b->retired.size() > 16);
}

// Launch the batch graph on s and record its event after the launch.
cudaError_t launch_batch_graph(kgs_batch* b, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (!b->graph_ev) e = cudaEventCreateWithFlags(&b->graph_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->graph_ev, s);
    return e;
}

// first-fit placement in the arena (256-byte aligned ranges)
bool arena_alloc(kgs_batch* b, size_t bytes, size_t* off)
{
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = b->free_ranges.begin(); it != b->free_ranges.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t roff = it->first + bytes;
            b->free_ranges.erase(it);
            if (rest) b->free_ranges[roff] = rest;
            return true;
        }
    }
    return false;
}

void arena_free(kgs_batch* b, size_t off, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    auto it = b->free_ranges.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != b->free_ranges.end() && it->first + it->second == next->first) {
        it->second += next->second;
        b->free_ranges.erase(next);
    }
    if (it != b->free_ranges.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            b->free_ranges.erase(it);
        }
    }
}

Coef<double> coef64(const HostInst& h)
{
    return host_coef64(h.dim, h.N, h.L, h.kappa1, h.kappa2, h.mu, h.gamma, h.tau);
}

Coef<float> coef32(const HostInst& h) { return host_coef32(coef64(h)); }

// Instances of one precision and dimension taking part in a call, in
// instance order, with the instance of every chunk and the pass at which each
// instance ends (2 n_i: its RED_ADJ pass).
template <typename T> struct HostList {
    std::vector<BatchInst<T>> inst;
    std::vector<int32_t> chunk_inst;
    std::vector<int64_t> ends;
    int64_t chunks = 0;
    bool wide = false;  // an instance has 2^31 points or more: 64-bit indices
};

template <typename T>
void build_lists(kgs_batch* b, const int64_t* nsteps, HostList<T> (&L)[3])
{
    const int prec = sizeof(T) == 8 ? 64 : 32;
    for (auto& l : L) l = HostList<T>();
    for (size_t i = 0; i < b->inst.size(); ++i) {
        const HostInst& h = b->inst[i];
        if (!h.live || h.precision != prec || nsteps[i] <= 0) continue;
        HostList<T>& l = L[h.dim - 1];
        BatchInst<T> d;
        d.pq = reinterpret_cast<vec2_t<T>*>(b->arena + h.off);
        d.uv = d.pq + h.M;
        d.dim = h.dim;
        d.N = (int)h.N;
        d.half = h.M / 2;
        d.first_chunk = l.chunks;
        d.nsteps = nsteps[i];
        if constexpr (sizeof(T) == 8) d.coef = coef64(h);
        else d.coef = coef32(h);
        const int64_t c = (d.half + kChunk - 1) / kChunk;
        l.chunk_inst.insert(l.chunk_inst.end(), (size_t)c, (int32_t)l.inst.size());
        l.inst.push_back(d);
        l.ends.push_back(2 * nsteps[i]);
        l.chunks += c;
        l.wide = l.wide || h.M >= ((int64_t)1 << 31);
    }
}

template <typename T>
int upload_list(kgs_batch* b, kgs_batch::DevList& dl, const HostList<T>& l, cudaStream_t s)
{
    if (l.inst.empty()) return KGS_OK;
    if ((int)l.inst.size() > dl.cap) {
        cudaFree(dl.inst);
        dl.inst = nullptr;
        dl.cap = 0;
        const int want = std::max<int>((int)l.inst.size(), 64);
        cudaError_t e = cudaMalloc(&dl.inst, want * sizeof(BatchInst<T>));
        if (e != cudaSuccess) return bcuda(b, e, "batch descriptor allocation");
        dl.cap = want;
    }
    if (l.chunks > dl.chunk_cap) {
        cudaFree(dl.chunk_inst);
        dl.chunk_inst = nullptr;
        dl.chunk_cap = 0;
        cudaError_t e = cudaMalloc(&dl.chunk_inst, (size_t)l.chunks * sizeof(int32_t));
        if (e != cudaSuccess) return bcuda(b, e, "batch work list allocation");
        dl.chunk_cap = l.chunks;
    }
    cudaError_t e = cudaMemcpyAsync(dl.inst, l.inst.data(), l.inst.size() * sizeof(BatchInst<T>),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dl.chunk_inst, l.chunk_inst.data(), (size_t)l.chunks * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s);
    // the host vectors must outlive the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bcuda(b, e, "batch work list upload");
    return KGS_OK;
}

template <typename T, int D, int MODE>
int launch_one(kgs_batch* b, const kgs_batch::DevList& dl, int64_t chunks, bool wide, int64_t g,
               cudaStream_t s)
{
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    const int lc = b->ctas_list[sizeof(T) == 8 ? 0 : 1][D - 1];
    const int64_t grid = std::min<int64_t>(chunks, (int64_t)sms * (lc > 0 ? lc : b->ctas_per_sm));
    const BatchInst<T>* insts = reinterpret_cast<const BatchInst<T>*>(dl.inst);
    if (wide)
        batch_pass_kernel<T, D, MODE, int64_t><<<(unsigned)grid, kChunk, 0, s>>>(insts, dl.chunk_inst, chunks, g);
    else
        batch_pass_kernel<T, D, MODE, int32_t><<<(unsigned)grid, kChunk, 0, s>>>(insts, dl.chunk_inst, chunks, g);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return bcuda(b, e, "batch pass launch");
    b->launches += 1;
    return KGS_OK;
}

// Pass g of one list: one launch per pass mode that occurs among its instances.
template <typename T, int D>
int launch_list_pass(kgs_batch* b, const kgs_batch::DevList& dl, const HostList<T>& l, int64_t g,
                     cudaStream_t s)
{
    if (l.chunks == 0) return KGS_OK;
    bool later = false, ending = false;
    for (int64_t e : l.ends) {
        later = later || e > g;
        ending = ending || e == g;
    }
    if (g == 0) return launch_one<T, D, RED_BASE>(b, dl, l.chunks, l.wide, g, s);
    if (g & 1) return later ? launch_one<T, D, BLACK_FUSED>(b, dl, l.chunks, l.wide, g, s) : KGS_OK;
    int r = later ? launch_one<T, D, RED_FUSED>(b, dl, l.chunks, l.wide, g, s) : KGS_OK;
    if (!r && ending) r = launch_one<T, D, RED_ADJ>(b, dl, l.chunks, l.wide, g, s);
    return r;
}


// The persistent launch of pass 0 .. passes-1 of every list (the lists'
// descriptors already uploaded): the barrier zeroed on s, then one
// cooperative launch of as many CTAs as fit on the device at once.  Returns
// 0 or the failing call's cudaError_t (the caller decides whether it sticks).
int launch_persistent(kgs_batch* b, const int64_t (&lchunks)[6], int64_t passes, cudaStream_t s)
{
    PersistLists pl;
    for (int k = 0; k < 6; ++k) {
        const kgs_batch::DevList& dl = b->lists[k / 3][k % 3];
        pl.inst[k] = dl.inst;
        pl.chunk_inst[k] = dl.chunk_inst;
        pl.chunks[k] = lchunks[k];
    }
    pl.passes = passes;
    int sms = 148, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_persistent_kernel, kChunk, 0);
    if (e != cudaSuccess || per < 1) return (int)(e == cudaSuccess ? cudaErrorLaunchOutOfResources : e);
    int64_t total = 0;
    for (int64_t c : lchunks) total += c;
    const int64_t want = b->ctas_per_sm > 0 ? std::min<int64_t>(b->ctas_per_sm, per) : per;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(total, (int64_t)sms * want));
    const unsigned expected = grid + (unsigned)b->stall;
    e = cudaMemsetAsync(b->pbar, 0, sizeof(BatchBarrier), s);
    if (e != cudaSuccess) return (int)e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kChunk);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BatchBarrier* bar = b->pbar;
    int* err = b->perr;
    e = cudaLaunchKernelEx(&cfg, batch_persistent_kernel, pl, bar, expected, err);
    if (e != cudaSuccess) return (int)e;
    b->launches += 1;
    return 0;
}

int ensure_persistent(kgs_batch* b)
{
    if (b->pbar) return KGS_OK;
    cudaError_t e = cudaMalloc(&b->pbar, sizeof(BatchBarrier));
    if (e == cudaSuccess) e = cudaHostAlloc(&b->perr, sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->pbar);
        b->pbar = nullptr;
        b->perr = nullptr;
        return bfail(KGS_ERR_OOM, "persistent batch barrier: %s", cudaGetErrorString(e));
    }
    *(volatile int*)b->perr = 0;
    return KGS_OK;
}

int batch_run(kgs_batch* b, const int64_t* nsteps, cudaStream_t s)
{
    HostList<double> l64[3];
    HostList<float> l32[3];
    build_lists(b, nsteps, l64);
    build_lists(b, nsteps, l32);
    int64_t nmax = 0;
    for (size_t i = 0; i < b->inst.size(); ++i)
        if (b->inst[i].live) nmax = std::max(nmax, nsteps[i]);
    if (nmax == 0) return KGS_OK;
    const int64_t passes = 2 * nmax + 1;
    std::vector<int64_t> key(nsteps, nsteps + b->inst.size());
    for (size_t i = 0; i < b->inst.size(); ++i)
        if (!b->inst[i].live) key[i] = -1;
    reap_graphs(b, false);
    if (b->use_graph && b->graph && key == b->graph_key) {
        cudaError_t e = launch_batch_graph(b, s);
        if (e != cudaSuccess) return bcuda(b, e, "batch graph launch");
        b->launches += b->graph_launches;
        return KGS_OK;
    }
    int st = KGS_OK;
    for (int d = 0; d < 3 && !st; ++d) {
        st = upload_list(b, b->lists[0][d], l64[d], s);
        if (!st) st = upload_list(b, b->lists[1][d], l32[d], s);
    }
    if (st) return st;
    // Every non-empty list on its own stream: the first on the caller's, the
    // others on side streams forked from it; all join back before the call's
    // work completes.
    const int64_t lchunks[6] = {l64[0].chunks, l64[1].chunks, l64[2].chunks,
                                l32[0].chunks, l32[1].chunks, l32[2].chunks};
    int nactive = 0;
    for (int k = 0; k < 6; ++k) nactive += lchunks[k] > 0;
    if (nactive > 1 && !b->fork && !(b->persistent)) {
        cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return bcuda(b, e, "side streams");
    }
    bool wide = false;
    for (int d = 0; d < 3; ++d) wide = wide || l64[d].wide || l32[d].wide;
    const bool persist = b->persistent && !wide;  // 32-bit indices only
    if (persist && (st = ensure_persistent(b))) return st;
    auto issue = [&](cudaStream_t main) -> int {
        if (persist) {
            const int r = launch_persistent(b, lchunks, passes, main);
            return r ? bcuda(b, (cudaError_t)r, "persistent batch launch") : KGS_OK;
        }
        cudaStream_t ls[6];
        bool first = true;
        if (nactive > 1) {
            cudaError_t e = cudaEventRecord(b->fork, main);
            if (e != cudaSuccess) return bcuda(b, e, "fork");
        }
        for (int k = 0; k < 6; ++k) {
            ls[k] = main;
            if (!lchunks[k]) continue;
            if (first) {
                first = false;
                continue;
            }
            cudaError_t e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
            if (e != cudaSuccess) return bcuda(b, e, "fork");
            ls[k] = b->side[k];
        }
        int r = KGS_OK;
        for (int64_t g = 0; g < passes && !r; ++g) {
            r = launch_list_pass<double, 1>(b, b->lists[0][0], l64[0], g, ls[0]);
            if (!r) r = launch_list_pass<double, 2>(b, b->lists[0][1], l64[1], g, ls[1]);
            if (!r) r = launch_list_pass<double, 3>(b, b->lists[0][2], l64[2], g, ls[2]);
            if (!r) r = launch_list_pass<float, 1>(b, b->lists[1][0], l32[0], g, ls[3]);
            if (!r) r = launch_list_pass<float, 2>(b, b->lists[1][1], l32[1], g, ls[4]);
            if (!r) r = launch_list_pass<float, 3>(b, b->lists[1][2], l32[2], g, ls[5]);
        }
        if (r) return r;
        for (int k = 0; k < 6; ++k) {
            if (ls[k] == main) continue;
            cudaError_t e = cudaEventRecord(b->join[k], ls[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(main, b->join[k], 0);
            if (e != cudaSuccess) return bcuda(b, e, "join");
        }
        return KGS_OK;
    };
    if (!b->use_graph || (persist && b->persist_nograph)) return issue(s);
    if (persist) {
        // one cooperative launch in a graph; if this driver refuses to capture
        // it, launch it directly from now on (one launch per call either way)
        drop_batch_graph(b);
        if (!b->capture_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return bcuda(b, e, "cudaStreamCreate");
        }
        const int64_t before = b->launches;
        cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        const int r = e == cudaSuccess ? launch_persistent(b, lchunks, passes, b->capture_stream) : (int)e;
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) e = cudaStreamEndCapture(b->capture_stream, &graph);
        if (!r && e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        b->launches = before;
        if (r || e != cudaSuccess) {
            cudaGetLastError();
            b->graph = nullptr;
            b->persist_nograph = true;
            return issue(s);
        }
        b->graph_launches = 1;
        b->graph_key = key;
        e = launch_batch_graph(b, s);
        if (e != cudaSuccess) return bcuda(b, e, "batch graph launch");
        b->launches += 1;
        return KGS_OK;
    }
    drop_batch_graph(b);
    if (!b->capture_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamCreate");
    }
    cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamBeginCapture");
    const int64_t before = b->launches;
    st = issue(b->capture_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->capture_stream, &graph);
    b->graph_launches = b->launches - before;
    b->launches = before;
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bcuda(b, e, "cudaGraphInstantiate");
    }
    b->graph_key = key;
    e = launch_batch_graph(b, s);
    if (e != cudaSuccess) return bcuda(b, e, "batch graph launch");
    b->launches += b->graph_launches;
    return KGS_OK;
}

int inst_check(kgs_batch* b, int64_t id)
{
    if (id < 0 || id >= (int64_t)b->inst.size() || !b->inst[id].live)
        return bfail(KGS_ERR_ARG, "no live instance %lld", (long long)id);
    return KGS_OK;
}

}  // namespace

extern "C" {

kgs_batch_handle kgs_batch_create(int device, int64_t capacity_bytes)
{
    if (capacity_bytes < 4096) {
        bfail(KGS_ERR_ARG, "capacity must be at least 4096 bytes");
        return nullptr;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        bfail(KGS_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
        return nullptr;
    }
    if (device < 0 && cudaGetDevice(&device) != cudaSuccess) {
        bfail(KGS_ERR_CUDA, "cudaGetDevice failed");
        return nullptr;
    }
    if (device >= ndev) {
        bfail(KGS_ERR_ARG, "device %d out of range", device);
        return nullptr;
    }
    BatchDevGuard guard(device);
    kgs_batch* b = new (std::nothrow) kgs_batch();
    if (!b) {
        bfail(KGS_ERR_OOM, "host allocation failed");
        return nullptr;
    }
    b->device = device;
    b->capacity = ((size_t)capacity_bytes + 255) & ~(size_t)255;
    e = cudaMalloc(&b->arena, b->capacity);
    if (e == cudaSuccess) {
        b->scratch_blocks = invariants_blocks(3, (int64_t)1 << 20);
        e = cudaMalloc(&b->scratch, (size_t)b->scratch_blocks * 3 * sizeof(double));
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->out_dev, 3 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&b->out_host, 3 * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        bfail(e == cudaErrorMemoryAllocation ? KGS_ERR_OOM : KGS_ERR_CUDA,
              "batch arena of %lld bytes: %s", (long long)capacity_bytes, cudaGetErrorString(e));
        cudaFree(b->arena);
        cudaFree(b->scratch);
        cudaFree(b->pbar);
        if (b->perr) cudaFreeHost(b->perr);
        cudaFree(b->out_dev);
        if (b->out_host) cudaFreeHost(b->out_host);
        delete b;
        return nullptr;
    }
    b->free_ranges[0] = b->capacity;
    return b;
}

int64_t kgs_batch_add(kgs_batch_handle b, int dim, int64_t N, double L, double kappa1,
                      double kappa2, double mu, double gamma, double tau, int precision)
{
    int st = bcheck(b);
    if (st) return st;
    if (dim < 1 || dim > 3) return bfail(KGS_ERR_ARG, "dim must be 1, 2 or 3");
    if (N < 4 || (N & 1)) return bfail(KGS_ERR_ODD_N, "N must be even and >= 4");
    if (N > 65534 || (dim == 3 && N > 4096) || (dim == 1 && N > (1 << 30)))
        return bfail(KGS_ERR_RANGE, "N out of range");
    if (!std::isfinite(L) || L <= 0 || !std::isfinite(kappa1) || !std::isfinite(kappa2) ||
        !std::isfinite(mu) || !std::isfinite(gamma) || !std::isfinite(tau) || tau == 0.0)
        return bfail(KGS_ERR_ARG, "parameters must be finite, L > 0, tau != 0");
    if (precision != KGS_FP64 && precision != KGS_FP32)
        return bfail(KGS_ERR_ARG, "precision must be KGS_FP64 or KGS_FP32");
    HostInst h;
    h.live = true;
    h.dim = dim;
    h.N = N;
    h.M = 1;
    for (int a = 0; a < dim; ++a) h.M *= N;
    h.L = L;
    h.kappa1 = kappa1;
    h.kappa2 = kappa2;
    h.mu = mu;
    h.gamma = gamma;
    h.tau = tau;
    h.precision = precision;
    h.bytes = (size_t)h.M * 2 * (precision == 64 ? sizeof(double2) : sizeof(float2));
    if (!arena_alloc(b, h.bytes, &h.off))
        return bfail(KGS_ERR_OOM, "instance needs %zu bytes; the arena has no free range that large",
                     h.bytes);
    // reuse a dead slot index if any
    for (size_t i = 0; i < b->inst.size(); ++i)
        if (!b->inst[i].live) {
            b->inst[i] = h;
            drop_batch_graph(b);
            return (int64_t)i;
        }
    b->inst.push_back(h);
    drop_batch_graph(b);
    return (int64_t)b->inst.size() - 1;
}

int kgs_batch_remove(kgs_batch_handle b, int64_t id)
{
    int st = bcheck(b);
    if (st) return st;
    if ((st = inst_check(b, id))) return st;
    arena_free(b, b->inst[id].off, b->inst[id].bytes);
    b->inst[id].live = false;
    drop_batch_graph(b);
    return KGS_OK;
}

int64_t kgs_batch_free_bytes(kgs_batch_handle b)
{
    if (!b) return bfail(KGS_ERR_ARG, "NULL batch handle");
    size_t best = 0;
    for (auto& r : b->free_ranges) best = std::max(best, r.second);
    return (int64_t)best;
}

int kgs_batch_set_state(kgs_batch_handle b, int64_t id, const double* P, const double* Q,
                        const double* U, const double* V, int where, void* stream)
{
    int st = bcheck(b);
    if (st) return st;
    if ((st = inst_check(b, id))) return st;
    if (!P || !Q || !U || !V || (where != KGS_HOST && where != KGS_DEVICE))
        return bfail(KGS_ERR_ARG, "NULL state pointer or bad memory kind");
    BatchDevGuard guard(b->device);
    HostInst& h = b->inst[id];
    cudaStream_t s = (cudaStream_t)stream;
    const double* src[4] = {P, Q, U, V};
    double* stage = nullptr;
    if (where == KGS_HOST) {
        cudaError_t e = cudaMallocAsync(&stage, (size_t)h.M * sizeof(double), s);
        if (e != cudaSuccess) return bcuda(b, e, "staging allocation");
    }
    for (int f = 0; f < 4; ++f) {
        const double* d = src[f];
        if (where == KGS_HOST) {
            cudaError_t e = cudaMemcpyAsync(stage, src[f], (size_t)h.M * sizeof(double),
                                            cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return bcuda(b, e, "state upload");
            d = stage;
        }
        char* base = b->arena + h.off;
        int n;
        if (h.precision == 64) {
            double2* dst = reinterpret_cast<double2*>(base) + (f < 2 ? 0 : h.M);
            n = launch_pack<double>(h.M, dst, f & 1, d, s, h.dim, h.N, f >= 2);
        } else {
            float2* dst = reinterpret_cast<float2*>(base) + (f < 2 ? 0 : h.M);
            n = launch_pack<float>(h.M, dst, f & 1, d, s, h.dim, h.N, f >= 2);
        }
        if (n < 0) return bcuda(b, cudaGetLastError(), "pack launch");
        b->launches += n;
    }
    if (where == KGS_HOST) {
        cudaFreeAsync(stage, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
    }
    h.state_set = true;
    return KGS_OK;
}

int kgs_batch_get_state(kgs_batch_handle b, int64_t id, double* P, double* Q, double* U, double* V,
                        int where, void* stream)
{
    int st = bcheck(b);
    if (st) return st;
    if ((st = inst_check(b, id))) return st;
    if (!P || !Q || !U || !V || (where != KGS_HOST && where != KGS_DEVICE))
        return bfail(KGS_ERR_ARG, "NULL state pointer or bad memory kind");
    BatchDevGuard guard(b->device);
    HostInst& h = b->inst[id];
    if (!h.state_set) return bfail(KGS_ERR_STATE, "instance has no state");
    cudaStream_t s = (cudaStream_t)stream;
    double* dst[4] = {P, Q, U, V};
    double* stage = nullptr;
    if (where == KGS_HOST) {
        cudaError_t e = cudaMallocAsync(&stage, (size_t)h.M * sizeof(double), s);
        if (e != cudaSuccess) return bcuda(b, e, "staging allocation");
    }
    for (int f = 0; f < 4; ++f) {
        double* d = (where == KGS_HOST) ? stage : dst[f];
        const char* base = b->arena + h.off;
        int n;
        if (h.precision == 64) {
            const double2* src = reinterpret_cast<const double2*>(base) + (f < 2 ? 0 : h.M);
            n = launch_unpack<double>(h.M, d, src, f & 1, s, h.dim, h.N, f >= 2);
        } else {
            const float2* src = reinterpret_cast<const float2*>(base) + (f < 2 ? 0 : h.M);
            n = launch_unpack<float>(h.M, d, src, f & 1, s, h.dim, h.N, f >= 2);
        }
        if (n < 0) return bcuda(b, cudaGetLastError(), "unpack launch");
        b->launches += n;
        if (where == KGS_HOST) {
            cudaError_t e = cudaMemcpyAsync(dst[f], stage, (size_t)h.M * sizeof(double),
                                            cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return bcuda(b, e, "state download");
        }
    }
    if (where == KGS_HOST) {
        cudaFreeAsync(stage, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
        return bcheck(b);  // a persistent launch before it may have timed out
    }
    return KGS_OK;
}

int kgs_batch_step_each(kgs_batch_handle b, const int64_t* nsteps, void* stream)
{
    NvtxRange range("kgs_batch_step");
    int st = bcheck(b);
    if (st) return st;
    if (!nsteps) return bfail(KGS_ERR_ARG, "NULL step counts");
    for (size_t i = 0; i < b->inst.size(); ++i) {
        if (!b->inst[i].live) continue;
        if (nsteps[i] < 0) return bfail(KGS_ERR_ARG, "negative step count for instance %zu", i);
        if (nsteps[i] > 0 && !b->inst[i].state_set)
            return bfail(KGS_ERR_STATE, "instance %zu has no state", i);
    }
    BatchDevGuard guard(b->device);
    return batch_run(b, nsteps, (cudaStream_t)stream);
}

int kgs_batch_step(kgs_batch_handle b, int64_t nsteps, void* stream)
{
    int st = bcheck(b);
    if (st) return st;
    if (nsteps < 0) return bfail(KGS_ERR_ARG, "nsteps must be >= 0");
    std::vector<int64_t> n(b->inst.size(), nsteps);
    for (size_t i = 0; i < b->inst.size(); ++i)
        if (!b->inst[i].live) n[i] = 0;
    return kgs_batch_step_each(b, n.data(), stream);
}

int kgs_batch_invariants(kgs_batch_handle b, int64_t id, double* out3, void* stream)
{
    NvtxRange range("kgs_batch_invariants");
    int st = bcheck(b);
    if (st) return st;
    if ((st = inst_check(b, id))) return st;
    if (!out3) return bfail(KGS_ERR_ARG, "NULL output");
    HostInst& h = b->inst[id];
    if (!h.state_set) return bfail(KGS_ERR_STATE, "instance has no state");
    BatchDevGuard guard(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    const InvParams p = make_inv_params(h.dim, h.L / (double)h.N, h.kappa1, h.kappa2, h.mu, h.gamma);
    Grid g{h.dim, h.N, h.M};
    g.split = true;
    const int nb = invariants_blocks(h.dim, h.N);
    const char* base = b->arena + h.off;
    int n = (h.precision == 64)
                ? launch_invariants<double>(g, reinterpret_cast<const double2*>(base),
                                            reinterpret_cast<const double2*>(base) + h.M, p,
                                            b->scratch, nb, b->out_dev, s)
                : launch_invariants<float>(g, reinterpret_cast<const float2*>(base),
                                           reinterpret_cast<const float2*>(base) + h.M, p,
                                           b->scratch, nb, b->out_dev, s);
    if (n < 0) return bcuda(b, cudaGetLastError(), "invariants launch");
    b->launches += n;
    cudaError_t e = cudaMemcpyAsync(b->out_host, b->out_dev, 3 * sizeof(double),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bcuda(b, e, "invariants readback");
    if ((st = bcheck(b))) return st;  // a persistent launch before it may have timed out
    for (int k = 0; k < 3; ++k) out3[k] = b->out_host[k];
    return KGS_OK;
}

int kgs_batch_set_option(kgs_batch_handle b, int option, int64_t value)
{
    int st = bcheck(b);
    if (st) return st;
    switch (option) {
    case KGS_BATCH_OPT_CTAS_PER_SM:
        if (value < 1 || value > 32) return bfail(KGS_ERR_ARG, "CTAs per SM take 1..32");
        b->ctas_per_sm = (int)value;
        for (auto& row : b->ctas_list)
            for (int& c : row) c = 0;
        drop_batch_graph(b);
        return KGS_OK;
    case KGS_BATCH_OPT_CTAS_LIST + 0:
    case KGS_BATCH_OPT_CTAS_LIST + 1:
    case KGS_BATCH_OPT_CTAS_LIST + 2:
    case KGS_BATCH_OPT_CTAS_LIST + 3:
    case KGS_BATCH_OPT_CTAS_LIST + 4:
    case KGS_BATCH_OPT_CTAS_LIST + 5: {
        if (value < 0 || value > 32) return bfail(KGS_ERR_ARG, "CTAs per SM of a list take 0..32");
        const int k = option - KGS_BATCH_OPT_CTAS_LIST;
        b->ctas_list[k / 3][k % 3] = (int)value;
        drop_batch_graph(b);
        return KGS_OK;
    }
    case KGS_BATCH_OPT_GRAPH:
        if (value < 0 || value > 1) return bfail(KGS_ERR_ARG, "graph option takes 0 or 1");
        b->use_graph = (int)value;
        drop_batch_graph(b);
        return KGS_OK;
    case KGS_BATCH_OPT_PERSISTENT:
        if (value < 0 || value > 1) return bfail(KGS_ERR_ARG, "persistent option takes 0 or 1");
        b->persistent = (int)value;
        drop_batch_graph(b);
        return KGS_OK;
    case KGS_BATCH_OPT_TEST_STALL:
        if (value < 0 || value > 1024) return bfail(KGS_ERR_ARG, "stall test hook takes 0 to 1024");
        b->stall = (int)value;
        drop_batch_graph(b);
        return KGS_OK;
    default:
        return bfail(KGS_ERR_ARG, "unknown batch option %d", option);
    }
}

int64_t kgs_batch_launch_count(kgs_batch_handle b) { return b ? b->launches : -1; }

void kgs_batch_destroy(kgs_batch_handle b)
{
    if (!b) return;
    {
        BatchDevGuard guard(b->device);
        cudaDeviceSynchronize();  // no queued work may still use what is freed below
        drop_batch_graph(b);
        reap_graphs(b, true);
        if (b->graph_ev) cudaEventDestroy(b->graph_ev);
        if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
        for (int k = 0; k < 6; ++k) {
            if (b->side[k]) cudaStreamDestroy(b->side[k]);
            if (b->join[k]) cudaEventDestroy(b->join[k]);
        }
        if (b->fork) cudaEventDestroy(b->fork);
        cudaFree(b->arena);
        for (auto& row : b->lists)
            for (auto& dl : row) {
                cudaFree(dl.inst);
                cudaFree(dl.chunk_inst);
            }
        cudaFree(b->scratch);
        cudaFree(b->out_dev);
        if (b->out_host) cudaFreeHost(b->out_host);
    }
    delete b;
}

}  // extern "C"
