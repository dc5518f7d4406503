// Persistent pipelined kernel of the packed FP32 path.
//
// One launch runs the four stages of the packed path (spread, column DFTs, row
// FFTs, epilogue; packed_stages.cuh) for a list of tasks, a task being one
// signal of one plan.  Tasks may come from different plans (uneven batches).
// Each stage of a task is cut into work items:
//   S  one 256-cell spread tile                       (ntiles items)
//   C  cm passes over 256 / cgw columns of one pair  (Kp * 4 cgw / cm items)
//   R  up to 8 rows of one taper pair                 (Kp * ceil(n1 / 8) items)
//   E  one 32 x 16 epilogue tile                      (epi_tiles(n1, k2max, 32) items)
// A host-built item list orders the items in rounds: round t holds the E items
// of task t - 3L, the R items of task t - 2L, the C items of task t - L and the
// S items of task t, so stages of different signals run side by side (compute-
// bound FFT items next to HBM-bound epilogue items) and the intermediates of a
// task (g, Z) are consumed a few rounds after they are written, while they
// are still in L2.  Task t uses workspace slot t mod ring.
//
// Scheduling: CTAs claim items in list order with one atomic counter and run
// them one at a time.  An item first waits until the stage it depends on is
// complete (per-task, per-stage completion counters):
//   S(t) <- E(t - ring) (slot reuse),  C(t) <- S(t),  R(t) <- C(t),  E(t) <- R(t).
// The host checks that every dependency lies strictly earlier in the list, so
// the lowest unfinished item always has its dependencies met and is held by a
// running CTA: the schedule cannot deadlock, whatever the number of resident
// CTAs.  Waits are still bounded (wall-clock limit via %globaltimer plus an
// iteration cap); on expiry the kernel raises an abort flag that every waiting
// CTA sees, records M2_ERR_TIMEOUT and the item, and all CTAs return.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "packed_stages.cuh"

namespace m2 {
namespace {

using packed::Ctx;
using packed::Tw32;
using packed::kRowLen;

constexpr int kPipeThreads = 256;
constexpr int kRowsPerItem = 8;
constexpr int kSpinCap = 1 << 24;  // iteration cap of one wait (the wall-clock limit normally ends it first)

enum : int { kStageS = 0, kStageC = 1, kStageR = 2, kStageE = 3 };
// control words in front of the completion counters
enum : int { kCtrlNext = 0, kCtrlAbort = 1, kCtrlStatus = 2, kCtrlItem = 3, kCtrlWords = 4 };

struct __align__(16) PipeTask {
    const float* x;
    float2* J;
    float* E;
    float* P;
    int ctx;
    int slot;
    int pad0, pad1;
};

struct __align__(16) PipeItem {
    int task;
    int ctx;
    int code;    // stage << 28 | index within the stage
    int dep;     // completion counter this item waits for, or -1
    int target;  // value the counter must reach
    int pad0, pad1, pad2;
};

static_assert(sizeof(Ctx) % 16 == 0 && sizeof(Ctx) <= 16 * 28, "Ctx is copied to shared memory as int4");
static_assert(sizeof(PipeTask) == 48, "PipeTask layout");
static_assert(sizeof(PipeItem) == 32, "PipeItem layout");

struct PipeArgs {
    const PipeItem* items;
    int nitems;
    const PipeTask* tasks;  // NULL: strided tasks of ctx 0 (x + t * sx, ...)
    const float* x0;
    float2* J0;
    float* E0;
    float* P0;
    int64_t sx, sJ, sP;  // strides of the strided form (elements)
    int ring;
    const Ctx* ctxs;
    float2* wg;  // workspace slots
    float2* wz;
    int64_t sg, sz;  // slot strides (float2)
    int* ctrl;            // [kCtrlWords] then [ntasks][4] completion counters
    int* hstat;           // mapped pinned [abort, status, item]: written when a wait gives up
    unsigned long long* prof;  // NULL, or per stage: [0..3] busy ns, [4..7] items, [8..11] wait ns
    long long timeout_ns;
    Tw32 tw;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long globaltimer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0: wait until *c >= target.  false = gave up (time limit, iteration cap, or another CTA's abort).
__device__ bool wait_counter(const int* c, int target, int* ctrl, int* hstat, long long timeout_ns, int item) {
    if (ld_acquire(c) >= target) return true;
    const long long t0 = globaltimer();
    for (int it = 0; it < kSpinCap; ++it) {
        __nanosleep(128);
        if (ld_acquire(c) >= target) return true;
        if (*(volatile int*)(ctrl + kCtrlAbort)) return false;
        if (globaltimer() - t0 > timeout_ns) break;
    }
    if (atomicCAS(ctrl + kCtrlStatus, 0, (int)M2_ERR_TIMEOUT) == 0) {
        ctrl[kCtrlItem] = item;
        volatile int* h = hstat;
        h[2] = item;
        h[1] = (int)M2_ERR_TIMEOUT;
        h[0] = 1;
        __threadfence_system();
    }
    atomicExch(ctrl + kCtrlAbort, 1);
    return false;
}

template <int F>
__device__ __forceinline__ void run_cols(const Ctx& c, const Tw32& tw, const float2* gb, float2* Zb, int idx,
                                         float2* smem) {
    // item idx: pair j, columns [cb * cm * P, (cb + 1) * cm * P) with P = 32 * 8 / cgw per pass
    const int gw = c.cgw, ngroups = 8 / gw;
    const int per_pair = 4 * gw / c.cm;
    const int j = idx / per_pair, cb = idx - j * per_pair;
    float2* s_tw = smem;  // [n1]
    const int warp = threadIdx.x >> 5;
    const int grp = warp / gw, gwarp = warp - grp * gw;
    float2* s_grp = smem + c.n1 + (size_t)grp * packed::cols_group_f2(false, c.rows, F, c.n1);
    packed::fill_n1_twiddles(c, s_tw);
    const float2* gj = gb + (int64_t)j * c.Lg;
    float2* Zj = Zb + (int64_t)j * c.n1 * kRowLen;
    for (int m = 0; m < c.cm; ++m) {
        const int colbase = ((cb * c.cm + m) * ngroups + grp) * 32;
        packed::cols_group<F, false>(c, tw, gj, Zj, colbase, gwarp, gw, s_tw, s_grp);
    }
}

__device__ __forceinline__ void stage_spread(const Ctx& c, const float* x, int idx, float2* gb, unsigned char* smem) {
    if (c.Kp <= 2) packed::spread_ell<2, 1>(c, x, 1, idx, gb, smem);
    else if (c.Kp <= 4) packed::spread_ell<4, 1>(c, x, 1, idx, gb, smem);
    else packed::spread_ell<8, 1>(c, x, 1, idx, gb, smem);
}

__device__ __forceinline__ void stage_cols(const Ctx& c, const Tw32& tw, const float2* gb, float2* Zb, int idx,
                                        float2* sm) {
    switch (c.F) {
        case 2: run_cols<2>(c, tw, gb, Zb, idx, sm); break;
        case 4: run_cols<4>(c, tw, gb, Zb, idx, sm); break;
        case 8: run_cols<8>(c, tw, gb, Zb, idx, sm); break;
        case 16: run_cols<16>(c, tw, gb, Zb, idx, sm); break;
        default: run_cols<32>(c, tw, gb, Zb, idx, sm); break;
    }
}

// Kept out of line: the row FFT needs all 128 registers the kernel's occupancy of two
// CTAs per SM allows, and inlined next to the column stage it spills far more.
__device__ __noinline__ void stage_rows(const Ctx& c, const Tw32& tw, float2* Zb, int idx, float2* sm) {
    const int nrb = (c.n1 + kRowsPerItem - 1) / kRowsPerItem;
    const int j = idx / nrb, rb = idx - j * nrb;
    const int r0 = rb * kRowsPerItem;
    const int64_t plane = (int64_t)c.n1 * kRowLen;
    packed::rowfft_rows<kRowsPerItem, false>(c, tw, Zb + j * plane, r0, min(kRowsPerItem, c.n1 - r0), sm);
}

// one 32 x 16 epilogue tile per item (L2-coherent loads; no discards: the ring slot is reused)
__device__ __forceinline__ void stage_epi(const Ctx& c, const float2* Zb, int idx, float2* J, float* E, float* P,
                                          float2* sm) {
    packed::epi_tile<32, kPipeThreads, false, false, false>(c, Zb, idx, J, E, P, nullptr, sm);
}

__global__ void __launch_bounds__(kPipeThreads, 2) pipe_kernel(PipeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) Ctx s_ctx;
    __shared__ __align__(16) PipeTask s_task;
    __shared__ int s_code, s_task_id, s_stop;
    // instrumentation (thread 0): item start (before the wait), end of the wait, and per-stage
    // sums of busy ns, items and wait ns, added to a.prof once when the CTA exits
    __shared__ long long s_t0, s_t1;
    __shared__ unsigned long long s_prof[12];
    const int tid = threadIdx.x;
    if (tid < 12) s_prof[tid] = 0;
    int ctx_loaded = -1;  // warp 0: context currently in s_ctx

    for (;;) {
        // ---- warp 0: claim the next item in list order (a CTA holds one item at a time, so no
        // item waits behind another while CTAs are idle), stage its task and context, and let
        // lane 0 wait for its dependency
        if (tid < 32) {
            int n = 0;
            if (tid == 0) n = atomicAdd(a.ctrl + kCtrlNext, 1);
            n = __shfl_sync(0xffffffffu, n, 0);
            if (n >= a.nitems) {
                if (tid == 0) s_stop = 1;
            } else {
                int4 dv = make_int4(0, 0, 0, 0);
                if (tid < 2) dv = reinterpret_cast<const int4*>(a.items + n)[tid];
                const int task = __shfl_sync(0xffffffffu, dv.x, 0);
                const int ctx = __shfl_sync(0xffffffffu, dv.y, 0);
                const int code = __shfl_sync(0xffffffffu, dv.z, 0);
                const int dep = __shfl_sync(0xffffffffu, dv.w, 0);
                const int target = __shfl_sync(0xffffffffu, dv.x, 1);
                if (tid >= 1 && tid <= 3) {
                    if (a.tasks) {
                        reinterpret_cast<int4*>(&s_task)[tid - 1] =
                            reinterpret_cast<const int4*>(a.tasks + task)[tid - 1];
                    } else if (tid == 1) {
                        s_task.x = a.x0 + (int64_t)task * a.sx;
                        s_task.J = a.J0 ? a.J0 + (int64_t)task * a.sJ : nullptr;
                        s_task.E = a.E0 ? a.E0 + (int64_t)task * a.sJ : nullptr;
                        s_task.P = a.P0 ? a.P0 + (int64_t)task * a.sP : nullptr;
                        s_task.ctx = 0;
                        s_task.slot = task % a.ring;
                    }
                } else if (ctx != ctx_loaded && tid >= 4 && tid - 4 < (int)(sizeof(Ctx) / 16)) {
                    reinterpret_cast<int4*>(&s_ctx)[tid - 4] = reinterpret_cast<const int4*>(a.ctxs + ctx)[tid - 4];
                }
                ctx_loaded = ctx;
                if (tid == 0) {
                    int stop = 0;
                    s_t0 = globaltimer();
                    if (dep >= 0 && !wait_counter(a.ctrl + kCtrlWords + dep, target, a.ctrl, a.hstat, a.timeout_ns, n))
                        stop = 2;
                    s_stop = stop;
                    s_code = code;
                    s_task_id = task;
                    s_t1 = globaltimer();
                }
            }
        }
        __syncthreads();
        if (s_stop) break;

        const Ctx& c = s_ctx;
        const int stage = s_code >> 28;
        const int idx = s_code & 0x0fffffff;
        const int slot = s_task.slot;
        float2* gb = a.wg + (int64_t)slot * a.sg;
        float2* Zb = a.wz + (int64_t)slot * a.sz;
        float2* sm = reinterpret_cast<float2*>(smem);
        if (stage == kStageS) stage_spread(c, s_task.x, idx, gb, smem);
        else if (stage == kStageC) stage_cols(c, a.tw, gb, Zb, idx, sm);
        else if (stage == kStageR) stage_rows(c, a.tw, Zb, idx, sm);
        else stage_epi(c, Zb, idx, s_task.J, s_task.E, s_task.P, sm);
        // publish completion: the data of S, C and R items is read by other CTAs (fence first);
        // E items only have to have finished reading their slot
        if (stage != kStageE) __threadfence();
        __syncthreads();
        if (tid == 0) {
            red_release_add(a.ctrl + kCtrlWords + s_task_id * 4 + stage, 1);
            const long long t2 = globaltimer();
            s_prof[stage] += (unsigned long long)(t2 - s_t1);
            s_prof[4 + stage] += 1ull;
            s_prof[8 + stage] += (unsigned long long)(s_t1 - s_t0);
        }
    }
    if (a.prof && tid < 12 && s_prof[tid]) atomicAdd(a.prof + tid, s_prof[tid]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct StageCounts {
    int n[4];
};

StageCounts stage_counts(const Ctx& c, int ntiles) {
    StageCounts s;
    s.n[kStageS] = ntiles;
    s.n[kStageC] = c.Kp * (4 * c.cgw / c.cm);
    s.n[kStageR] = c.Kp * ((c.n1 + kRowsPerItem - 1) / kRowsPerItem);
    s.n[kStageE] = packed::epi_tiles(c.n1, c.k2max, 32);
    return s;
}

size_t pipe_smem_bytes(const Ctx& c) {
    const size_t spread = packed::spread_ell_smem_bytes(c.Kp, 1, c.ecap, c.pcap, c.ncap);
    const size_t cols = sizeof(float2) * (packed::cols_tw_f2(false, c.n1, c.rows, c.F) +
                                          (size_t)(8 / c.cgw) * packed::cols_group_f2(false, c.rows, c.F, c.n1));
    const size_t rows = packed::rowfft_smem_bytes(kRowsPerItem);
    return std::max(spread, std::max(cols, rows));
}

// Items in rounds (see the file comment).  lag 0 runs the stages of a task back to back.
// Returns the smallest distance, in items, from the last item a stage block depends on to
// the block's first item (taken over the steady-state tasks when there are enough), or -1
// if some dependency does not precede its dependent item (such a list is never launched).
int64_t build_items(const std::vector<int>& task_ctx, const std::vector<StageCounts>& counts, int ring, int lag,
                    std::vector<PipeItem>& items) {
    const int T = (int)task_ctx.size();
    items.clear();
    std::vector<int64_t> first((size_t)T * 4, -1), last((size_t)T * 4, -1);
    auto emit = [&](int t, int stage) {
        if (t < 0 || t >= T) return;
        const int n = counts[t].n[stage];
        int dep = -1, target = 0;
        if (stage == kStageS) {
            if (t - ring >= 0) {
                dep = (t - ring) * 4 + kStageE;
                target = counts[t - ring].n[kStageE];
            }
        } else {
            dep = t * 4 + stage - 1;
            target = counts[t].n[stage - 1];
        }
        first[(size_t)t * 4 + stage] = (int64_t)items.size();
        for (int i = 0; i < n; ++i) items.push_back(PipeItem{t, task_ctx[t], (stage << 28) | i, dep, target, 0, 0, 0});
        last[(size_t)t * 4 + stage] = (int64_t)items.size() - 1;
    };
    for (int r = 0; r < T + 3 * lag; ++r) {
        if (lag == 0) {
            emit(r, kStageS);
            emit(r, kStageC);
            emit(r, kStageR);
            emit(r, kStageE);
        } else {
            emit(r - 3 * lag, kStageE);
            emit(r - 2 * lag, kStageR);
            emit(r - lag, kStageC);
            emit(r, kStageS);
        }
    }
    const bool steady = T > 6 * lag + 2;
    int64_t gap = INT64_MAX;
    for (int t = 0; t < T; ++t)
        for (int s = 0; s < 4; ++s) {
            const size_t k = (size_t)t * 4 + s;
            if (counts[t].n[s] <= 0 || first[k] < 0) return -1;
            int dk = -1;
            if (s == kStageS) {
                if (t - ring >= 0) dk = (t - ring) * 4 + kStageE;
            } else {
                dk = (int)k - 1;
            }
            if (dk < 0) continue;
            if (last[dk] >= first[k]) return -1;
            if (!steady || (t >= 3 * lag && t < T - 3 * lag)) gap = std::min(gap, first[k] - last[dk]);
        }
    return gap;
}

}  // namespace

// Device and host resources of one pipelined launch configuration.
struct PipeLaunch {
    int device = 0;
    int nitems = 0, ntasks = 0, ring = 1;
    int grid = 0;
    size_t smem = 0;
    PipeItem* d_items = nullptr;
    PipeTask* d_tasks = nullptr;  // NULL for the strided form
    Ctx* d_ctxs = nullptr;
    int* d_ctrl = nullptr;
    int* h_status = nullptr;  // mapped pinned [abort, status, item] (owned if own_status)
    int* d_status = nullptr;  // its device alias
    bool own_status = false;
    float2 *wg = nullptr, *wz = nullptr;
    int64_t sg = 0, sz = 0;
    unsigned long long* d_prof = nullptr;  // batch launches: stage accounting (owned), accumulated
    std::vector<void*> owned;  // device buffers owned by this launch
    Tw32 tw;

    ~PipeLaunch() {
        for (void* q : owned) cudaFree(q);
        if (own_status && h_status) cudaFreeHost(h_status);
    }
};

namespace {

constexpr long long kPipeTimeoutNs = 2000000000LL;  // 2 s per wait

m2_status alloc_status(int** h, int** d) {
    M2_CUDA_TRY(cudaHostAlloc(h, 4 * sizeof(int), cudaHostAllocMapped));
    std::memset(*h, 0, 4 * sizeof(int));
    M2_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(d), *h, 0));
    return M2_OK;
}

template <typename T>
m2_status upload(PipeLaunch& L, T** dst, const T* src, size_t n) {
    M2_CUDA_TRY(cudaMalloc(dst, n * sizeof(T)));
    L.owned.push_back(*dst);
    M2_CUDA_TRY(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return M2_OK;
}

// Item list, context table, counters and grid of a launch configuration.  The pipeline lag
// (and with it the workspace ring, 3 lag + 1 slots, at most max_ring) is the smallest that puts
// two grids' worth of items between every stage block and the block it waits for, so CTAs
// rarely wait; signals with few items each (small plans) get a deeper pipeline.
m2_status pipe_setup(PipeLaunch& L, const std::vector<Ctx>& ctxs, const std::vector<int>& task_ctx,
                     const std::vector<int64_t>& ntiles, int max_ring) {
    std::vector<StageCounts> counts(task_ctx.size());
    size_t smem = 0;
    for (size_t t = 0; t < task_ctx.size(); ++t) counts[t] = stage_counts(ctxs[task_ctx[t]], (int)ntiles[task_ctx[t]]);
    for (const Ctx& c : ctxs) smem = std::max(smem, pipe_smem_bytes(c));
    int per_sm = 0, sms = 0;
    M2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pipe_kernel, kPipeThreads, smem));
    M2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, L.device));
    if (per_sm < 1) {
        set_error("pipelined kernel does not fit an SM (%zu bytes of shared memory)", smem);
        return M2_ERR_ARG;
    }
    const int64_t want_gap = 2 * (int64_t)per_sm * sms;
    std::vector<PipeItem> items;
    int ring = 1, best_lag = -1;
    int64_t best_gap = -1;
    for (int lag = 0; 3 * lag + 1 <= std::max(max_ring, 1) && lag <= 16; ++lag) {
        const int r = lag == 0 ? std::min(max_ring, 2) : 3 * lag + 1;
        const int64_t gap = build_items(task_ctx, counts, std::max(r, 1), lag, items);
        if (gap > best_gap) {
            best_gap = gap;
            best_lag = lag;
            ring = std::max(r, 1);
        }
        if (gap >= want_gap) break;
    }
    if (best_lag < 0 || build_items(task_ctx, counts, ring, best_lag, items) < 0) {
        set_error("internal: pipelined schedule has a dependency that does not precede its item");
        return M2_ERR_ARG;
    }
    if (items.size() > (size_t)0x7fffffff / 2) {
        set_error("pipelined batch too large (%zu work items)", items.size());
        return M2_ERR_ARG;
    }
    L.nitems = (int)items.size();
    L.ntasks = (int)task_ctx.size();
    L.ring = ring;
    L.smem = smem;
    L.tw = packed::make_tw32();
    M2_TRY(upload(L, &L.d_items, items.data(), items.size()));
    M2_TRY(upload(L, &L.d_ctxs, ctxs.data(), ctxs.size()));
    M2_CUDA_TRY(cudaMalloc(&L.d_ctrl, sizeof(int) * (kCtrlWords + 4 * (size_t)L.ntasks)));
    L.owned.push_back(L.d_ctrl);
    L.grid = (int)std::min<int64_t>((int64_t)per_sm * sms, L.nitems);
    return M2_OK;
}

// Report (once) a wait that gave up in an earlier launch sharing this status word.
m2_status check_status(int* h) {
    if (h && ((volatile int*)h)[0] != 0) {
        const int item = h[2];
        h[0] = h[1] = h[2] = 0;
        set_error("an earlier pipelined launch gave up waiting at work item %d (M2_ERR_TIMEOUT)", item);
        return M2_ERR_TIMEOUT;
    }
    return M2_OK;
}

m2_status pipe_run(PipeLaunch& L, const float* x0, float2* J0, float* E0, float* P0, int64_t sx, int64_t sJ,
                   int64_t sP, long long timeout_ns, unsigned long long* prof, cudaStream_t st) {
    M2_CUDA_TRY(cudaMemsetAsync(L.d_ctrl, 0, sizeof(int) * (kCtrlWords + 4 * (size_t)L.ntasks), st));
    PipeArgs a;
    a.items = L.d_items;
    a.nitems = L.nitems;
    a.tasks = L.d_tasks;
    a.x0 = x0;
    a.J0 = J0;
    a.E0 = E0;
    a.P0 = P0;
    a.sx = sx;
    a.sJ = sJ;
    a.sP = sP;
    a.ring = L.ring;
    a.ctxs = L.d_ctxs;
    a.wg = L.wg;
    a.wz = L.wz;
    a.sg = L.sg;
    a.sz = L.sz;
    a.ctrl = L.d_ctrl;
    a.hstat = L.d_status;
    a.prof = prof;
    a.timeout_ns = timeout_ns;
    a.tw = L.tw;
    pipe_kernel<<<L.grid, kPipeThreads, L.smem, st>>>(a);
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

}  // namespace

void pipe_batch_forget(PipeLaunch* L);

void pipe_free(PipeLaunch* L) {
    pipe_batch_forget(L);
    delete L;
}

m2_status init_pipe_kernels(int smem_optin) {
    // the kernel's static shared memory counts against the per-block limit
    cudaFuncAttributes fa;
    M2_CUDA_TRY(cudaFuncGetAttributes(&fa, pipe_kernel));
    M2_CUDA_TRY(cudaFuncSetAttribute(pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem_optin - (int)fa.sharedSizeBytes));
    return M2_OK;
}

m2_status pipe_prepare(m2nufft_plan_s* p, int64_t B) {
    const Geometry& g = p->g;
    if (B < 1 || B > (int64_t)1 << 22) {
        set_error("m2nufft_exec: B = %lld out of range for one pipelined launch", (long long)B);
        return M2_ERR_ARG;
    }
    if (p->pipe_cache.count(B)) return M2_OK;
    if (!p->pipe_status) {
        int* d = nullptr;
        M2_TRY(alloc_status(&p->pipe_status, &d));
    }
    std::unique_ptr<PipeLaunch> nl(new PipeLaunch());
    nl->device = p->device;
    nl->h_status = p->pipe_status;
    M2_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&nl->d_status), p->pipe_status, 0));
    const Ctx c = packed_ctx(p);
    std::vector<int> task_ctx((size_t)B, 0);
    M2_TRY(pipe_setup(*nl, {c}, task_ctx, {g.ntiles}, g.chunk));  // ring slots: the plan's chunk workspace
    // ring slots: the plan's chunk workspace, slot s = signal s of a chunk
    nl->wg = reinterpret_cast<float2*>(p->d_g);
    nl->wz = reinterpret_cast<float2*>(p->d_Z);
    nl->sg = (int64_t)g.kp * g.Lg;
    nl->sz = (int64_t)g.kp * g.nf;
    p->pipe_cache.emplace(B, nl.release());
    return M2_OK;
}

// Single plan, B signals (strided): one launch.
m2_status exec_pipe(m2nufft_plan_s* p, const float* x, int64_t B, float2* J, float* E, float* P, cudaStream_t st) {
    const Geometry& g = p->g;
    M2_TRY(check_status(p->pipe_status));
    M2_TRY(pipe_prepare(p, B));
    PipeLaunch* L = p->pipe_cache.at(B);
    mark(p, 0, 0, st);
    if (p->timing && !p->d_pipe_prof) {
        M2_CUDA_TRY(cudaMalloc(&p->d_pipe_prof, 12 * sizeof(unsigned long long)));
        M2_CUDA_TRY(cudaMemset(p->d_pipe_prof, 0, 12 * sizeof(unsigned long long)));
    }
    M2_TRY(pipe_run(*L, x, J, E, P, g.N, (int64_t)g.K * g.I, g.I, kPipeTimeoutNs,
                    p->timing ? p->d_pipe_prof : nullptr, st));
    mark(p, 0, 1, st);
    return M2_OK;
}

// Uneven batch: signal s of plans[s] (packed FP32 plans of one device).
m2_status pipe_batch_create(m2nufft_plan_s* const* plans, const void* const* xs, int64_t nsig, void* const* Js,
                            void* const* Es, void* const* Ps, PipeLaunch** out) {
    std::unique_ptr<PipeLaunch> L(new PipeLaunch());
    L->device = plans[0]->device;
    M2_TRY(alloc_status(&L->h_status, &L->d_status));
    L->own_status = true;
    std::vector<Ctx> ctxs;
    std::vector<int64_t> ntiles;
    std::map<const m2nufft_plan_s*, int> index;
    std::vector<int> task_ctx((size_t)nsig);
    int64_t sg = 0, sz = 0;
    for (int64_t s = 0; s < nsig; ++s) {
        const m2nufft_plan_s* p = plans[s];
        auto f = index.find(p);
        if (f == index.end()) {
            f = index.emplace(p, (int)ctxs.size()).first;
            ctxs.push_back(packed_ctx(p));
            ntiles.push_back(p->g.ntiles);
            sg = std::max<int64_t>(sg, (int64_t)p->g.kp * p->g.Lg);
            sz = std::max<int64_t>(sz, (int64_t)p->g.kp * p->g.nf);
        }
        task_ctx[(size_t)s] = f->second;
    }
    // ring of at most 64 slots and 4 GiB of workspace
    const int64_t slot_bytes = (int64_t)sizeof(float2) * (sg + 2 * sz);
    const int max_ring = (int)std::max<int64_t>(1, std::min<int64_t>(64, (int64_t(4) << 30) / slot_bytes));
    M2_TRY(pipe_setup(*L, ctxs, task_ctx, ntiles, max_ring));
    const int ring = L->ring;
    std::vector<PipeTask> tasks((size_t)nsig);
    for (int64_t s = 0; s < nsig; ++s) {
        tasks[(size_t)s] = PipeTask{static_cast<const float*>(xs[s]), Js ? static_cast<float2*>(Js[s]) : nullptr,
                                    Es ? static_cast<float*>(Es[s]) : nullptr,
                                    Ps ? static_cast<float*>(Ps[s]) : nullptr, task_ctx[(size_t)s], (int)(s % ring),
                                    0, 0};
    }
    M2_TRY(upload(*L, &L->d_tasks, tasks.data(), tasks.size()));
    M2_CUDA_TRY(cudaMalloc(&L->d_prof, 12 * sizeof(unsigned long long)));
    L->owned.push_back(L->d_prof);
    M2_CUDA_TRY(cudaMemset(L->d_prof, 0, 12 * sizeof(unsigned long long)));
    // ring workspace: g and Z slots sized for the largest plan
    L->sg = sg;
    L->sz = sz;
    M2_CUDA_TRY(cudaMalloc(&L->wg, sizeof(float2) * (size_t)(sg * ring)));
    L->owned.push_back(L->wg);
    M2_CUDA_TRY(cudaMalloc(&L->wz, sizeof(float2) * (size_t)(sz * ring)));
    L->owned.push_back(L->wz);
    *out = L.release();
    return M2_OK;
}

m2_status pipe_check(PipeLaunch* L) { return check_status(L->h_status); }

namespace {
std::mutex g_batch_prof_mu;
PipeLaunch* g_last_batch = nullptr;  // most recently launched batch (stage accounting)
}  // namespace

m2_status pipe_batch_run(PipeLaunch* L, cudaStream_t st) {
    {
        std::lock_guard<std::mutex> lock(g_batch_prof_mu);
        g_last_batch = L;
    }
    return pipe_run(*L, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, kPipeTimeoutNs, L->d_prof, st);
}

void pipe_batch_mark_launched(PipeLaunch* L) {
    std::lock_guard<std::mutex> lock(g_batch_prof_mu);
    g_last_batch = L;
}

void pipe_batch_forget(PipeLaunch* L) {
    std::lock_guard<std::mutex> lock(g_batch_prof_mu);
    if (g_last_batch == L) g_last_batch = nullptr;
}

unsigned long long* pipe_last_batch_profile(int* device) {
    std::lock_guard<std::mutex> lock(g_batch_prof_mu);
    if (!g_last_batch) return nullptr;
    *device = g_last_batch->device;
    return g_last_batch->d_prof;
}

}  // namespace m2

// Bounded-wait self-test of the pipelined kernel: one work item waiting on a completion counter
// that nothing increments.  The wait gives up after timeout_ms, the kernel returns, and the
// status word reads M2_ERR_TIMEOUT at work item 0.
extern "C" m2_status m2nufft_pipe_selftest(int timeout_ms, void* stream) {
    using namespace m2;
    clear_error();
    if (timeout_ms < 1 || timeout_ms > 10000) {
        set_error("m2nufft_pipe_selftest: timeout_ms must be in [1, 10000]");
        return M2_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PipeLaunch L;
    M2_CUDA_TRY(cudaGetDevice(&L.device));
    M2_TRY(alloc_status(&L.h_status, &L.d_status));
    L.own_status = true;
    // one context and one task, read by the kernel but never used: zeros
    Ctx c;
    std::memset(&c, 0, sizeof(c));
    c.Kp = 1;
    c.n1 = 2;
    c.cm = 1;
    c.cgw = 4;
    c.F = 2;
    const PipeItem item{0, 0, kStageS << 28, 4 /* task 1, stage S: never incremented */, 1, 0, 0, 0};
    const PipeTask task{};
    L.nitems = 1;
    L.ntasks = 2;
    L.ring = 1;
    L.smem = pipe_smem_bytes(c);
    L.tw = packed::make_tw32();
    L.grid = 1;
    M2_TRY(upload(L, &L.d_items, &item, 1));
    M2_TRY(upload(L, &L.d_ctxs, &c, 1));
    M2_TRY(upload(L, &L.d_tasks, &task, 1));
    M2_CUDA_TRY(cudaMalloc(&L.d_ctrl, sizeof(int) * (kCtrlWords + 4 * (size_t)L.ntasks)));
    L.owned.push_back(L.d_ctrl);
    M2_TRY(init_device_kernels(L.device));
    M2_TRY(pipe_run(L, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, (long long)timeout_ms * 1000000LL, nullptr, st));
    M2_CUDA_TRY(cudaStreamSynchronize(st));
    const volatile int* h = L.h_status;
    if (h[0] == 1 && h[1] == (int)M2_ERR_TIMEOUT && h[2] == 0) {
        set_error("pipelined kernel gave up waiting at work item 0 as intended");
        return M2_ERR_TIMEOUT;
    }
    set_error("pipelined kernel self-test: unexpected status (abort %d, status %d, item %d)", h[0], h[1], h[2]);
    return M2_ERR_CUDA;
}

extern "C" m2_status m2nufft_get_pipe_profile(m2nufft_plan_t p, double* busy_ms, double* wait_ms, int64_t* items) {
    using namespace m2;
    clear_error();
    unsigned long long h[12] = {};
    int dev = 0;
    unsigned long long* src = nullptr;
    if (p) {
        src = p->d_pipe_prof;
        dev = p->device;
    } else {
        src = pipe_last_batch_profile(&dev);
    }
    if (src) {
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != dev) M2_CUDA_TRY(cudaSetDevice(dev));
        cudaError_t e = cudaMemcpy(h, src, sizeof(h), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemset(src, 0, sizeof(h));
        if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        M2_CUDA_TRY(e);
    }
    for (int k = 0; k < 4; ++k) {
        if (busy_ms) busy_ms[k] = 1e-6 * (double)h[k];
        if (items) items[k] = (int64_t)h[4 + k];
        if (wait_ms) wait_ms[k] = 1e-6 * (double)h[8 + k];
    }
    return M2_OK;
}
