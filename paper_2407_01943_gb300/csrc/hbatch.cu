// Stage-batched executor for uneven batches of packed FP32 plans.
//
// An uneven batch (signal s with its own plan p_s: own sampling times, N, K,
// I and FFT geometry) runs as one kernel launch per stage over all signals of
// the batch -- spread, column DFTs (one launch per coset FFT length F), row
// FFTs, epilogue -- each stage at the occupancy its own register and shared-
// memory needs allow, captured as one CUDA graph by m2nufft_exec_batch.  The
// stage bodies are those of packed_stages.cuh, so every signal's J, |J|^2 and
// P-hat are bit-identical to m2nufft_exec on its own plan.
//
// Every CTA reads one entry of a per-stage work map built on the host (task,
// and the stage's index within that task), then that task's record and its
// plan context; the intermediates of all signals live in one workspace
// (signal s at offsets g_off / z_off), so stages of different signals never
// wait on each other and the whole batch is four to eight launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "packed_stages.cuh"

namespace m2 {
namespace {

using packed::Ctx;
using packed::Tw32;
using packed::kRowLen;

constexpr int kColThreads = 128;  // 4 warps: one group of 4 warps, or 4 one-warp groups

struct __align__(16) HTask {
    const float* x;
    float2* J;
    float* E;
    float* P;
    int64_t g_off;  // spread grids [Kp][Lg] at ws + g_off
    int64_t z_off;  // Z [Kp][n1][1024] at ws + z_off (then, in place, the row transforms)
    int ctx;
    int pad0;
    float* F;  // Thomson F-statistic [I], or NULL
};
static_assert(sizeof(HTask) == 64, "HTask layout");

// CTA prologue: stage the task record and the plan context in shared memory
__device__ __forceinline__ void load_task(const HTask* tasks, const Ctx* ctxs, int task, HTask* s_task, Ctx* s_ctx) {
    const int t = threadIdx.x;
    if (t < 4) reinterpret_cast<int4*>(s_task)[t] = reinterpret_cast<const int4*>(tasks + task)[t];
    __syncthreads();
    if (t < (int)(sizeof(Ctx) / 16))
        reinterpret_cast<int4*>(s_ctx)[t] = reinterpret_cast<const int4*>(ctxs + s_task->ctx)[t];
    __syncthreads();
}

// map entry: (task, first tile, tiles); up to NT tiles per CTA, one after the other (the task
// prologue is amortised over them).  Dynamic smem: the largest spread_ell_smem_bytes(Kp, 1, ...) of the batch.
template <int KP, int NT>
__global__ void __launch_bounds__(kSpreadTile) hb_spread_kernel(const int4* __restrict__ map, const HTask* tasks,
                                                                const Ctx* ctxs, float2* ws) {
    extern __shared__ __align__(16) unsigned char smem_hb[];
    __shared__ __align__(16) Ctx s_ctx;
    __shared__ __align__(16) HTask s_task;
    const int4 m = map[blockIdx.x];
    load_task(tasks, ctxs, m.x, &s_task, &s_ctx);
#pragma unroll 1
    for (int u = 0; u < NT && u < m.z; ++u)
        packed::spread_ell<KP, 1>(s_ctx, s_task.x, 1, m.y + u, ws + s_task.g_off, smem_hb);
}

// map entry: (task, pair, first column, warps per 32-column group); the CTA's 4 warps form
// 4 / gw groups on consecutive 32-column blocks
template <int F>
__global__ void __launch_bounds__(kColThreads) hb_cols_kernel(const int4* __restrict__ map, const HTask* tasks,
                                                              const Ctx* ctxs, Tw32 tw, float2* ws) {
    extern __shared__ float2 smem_f2[];
    __shared__ __align__(16) Ctx s_ctx;
    __shared__ __align__(16) HTask s_task;
    const int4 m = map[blockIdx.x];
    load_task(tasks, ctxs, m.x, &s_task, &s_ctx);
    const Ctx& c = s_ctx;
    const int gw = m.w;
    const int warp = threadIdx.x >> 5;
    const int grp = warp / gw, gwarp = warp - grp * gw;
    float2* s_tw = smem_f2;  // [n1]
    packed::fill_n1_twiddles(c, s_tw);
    float2* ws_g = ws + s_task.g_off + (int64_t)m.y * c.Lg;
    float2* ws_z = ws + s_task.z_off + (int64_t)m.y * c.n1 * kRowLen;
    packed::cols_group<F, false>(c, tw, ws_g, ws_z, m.z + grp * 32, gwarp, gw, s_tw,
                                 s_tw + c.n1 + (size_t)grp * packed::cols_group_f2(false, c.rows, F, c.n1));
}

// map entry: (task, pair, first row, rows); one warp per row, R rows per CTA
template <int R>
__global__ void __launch_bounds__(32 * R, 16 / R) hb_rows_kernel(const int4* __restrict__ map, const HTask* tasks,
                                                                 const Ctx* ctxs, Tw32 tw, float2* ws) {
    extern __shared__ float2 smem_f2[];
    __shared__ __align__(16) Ctx s_ctx;
    __shared__ __align__(16) HTask s_task;
    const int4 m = map[blockIdx.x];
    load_task(tasks, ctxs, m.x, &s_task, &s_ctx);
    const Ctx& c = s_ctx;
    float2* Z = ws + s_task.z_off + (int64_t)m.y * c.n1 * kRowLen;
    packed::rowfft_rows<R, true>(c, tw, Z, m.z, m.w, smem_f2);
}

// map entry: (task, epilogue tile); the epilogue with the F-statistic: 16 x 16 tiles, 256 threads,
// one position per thread (the stage and tile shape of the four-kernel path's F epilogue, so the
// results are bit-identical to m2nufft_exec_ftest)
__global__ void __launch_bounds__(256, 4) hb_epi_f_kernel(const int2* __restrict__ map, const HTask* tasks,
                                                          const Ctx* ctxs, const float2* ws) {
    __shared__ __align__(16) Ctx s_ctx;
    __shared__ __align__(16) HTask s_task;
    __shared__ __align__(16) float2 smem[packed::epi_tile_smem_bytes(16) / sizeof(float2)];
    const int2 m = map[blockIdx.x];
    load_task(tasks, ctxs, m.x, &s_task, &s_ctx);
    packed::epi_tile<16, 256, true, true, true>(s_ctx, ws + s_task.z_off, m.y, s_task.J, s_task.E, s_task.P,
                                                s_task.F, smem);
}

// map entry: (task, epilogue tile); one T1 x 16 tile per CTA, one position per thread
template <int T1>
__global__ void __launch_bounds__(16 * T1) hb_epi_kernel(const int2* __restrict__ map, const HTask* tasks,
                                                         const Ctx* ctxs, const float2* ws) {
    __shared__ __align__(16) Ctx s_ctx;
    __shared__ __align__(16) HTask s_task;
    __shared__ __align__(16) float2 smem[packed::epi_tile_smem_bytes(T1) / sizeof(float2)];
    const int2 m = map[blockIdx.x];
    load_task(tasks, ctxs, m.x, &s_task, &s_ctx);
    packed::epi_tile<T1, 16 * T1, true, false, true>(s_ctx, ws + s_task.z_off, m.y, s_task.J, s_task.E, s_task.P,
                                                     nullptr, smem);
}

template <typename T>
m2_status upload_vec(std::vector<void*>& owned, T** dst, const std::vector<T>& v) {
    *dst = nullptr;
    if (v.empty()) return M2_OK;
    M2_CUDA_TRY(cudaMalloc(dst, v.size() * sizeof(T)));
    owned.push_back(*dst);
    M2_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return M2_OK;
}

}  // namespace

// Resources of one uneven batch (owned by the cached batch graph).
struct HBatch {
    int device = 0;
    HBConfig cfg;
    std::vector<void*> owned;
    Ctx* d_ctxs = nullptr;
    HTask* d_tasks = nullptr;
    float2* ws = nullptr;
    Tw32 tw;
    int4* d_spread[3] = {};  // KP = 2, 4, 8
    int n_spread[3] = {};
    int4* d_cols[6] = {};  // F = 1 (unused), 2, 4, 8, 16, 32 by log2
    int n_cols[6] = {};
    size_t smem_cols[6] = {};
    int4* d_rows = nullptr;
    int n_rows = 0;
    int2* d_epi[3] = {};  // epilogue tile heights 8, 16, 32
    int n_epi[3] = {};
    int2* d_epif = nullptr;  // epilogue with the F-statistic
    int n_epif = 0;
    size_t ws_bytes = 0;
    size_t spread_smem = 0;

    ~HBatch() {
        for (void* q : owned) cudaFree(q);
    }
};

void hbatch_free(HBatch* h) { delete h; }

m2_status init_hbatch_kernels(int smem_optin) {
    const void* funcs[] = {(const void*)hb_cols_kernel<2>,  (const void*)hb_cols_kernel<4>,
                           (const void*)hb_cols_kernel<8>,  (const void*)hb_cols_kernel<16>,
                           (const void*)hb_cols_kernel<32>, (const void*)hb_rows_kernel<4>,
                           (const void*)hb_rows_kernel<8>};
    const void* spread[] = {
        (const void*)hb_spread_kernel<2, 1>, (const void*)hb_spread_kernel<2, 2>, (const void*)hb_spread_kernel<2, 4>,
        (const void*)hb_spread_kernel<4, 1>, (const void*)hb_spread_kernel<4, 2>, (const void*)hb_spread_kernel<4, 4>,
        (const void*)hb_spread_kernel<8, 1>, (const void*)hb_spread_kernel<8, 2>, (const void*)hb_spread_kernel<8, 4>,
    };
    for (const void* f : spread) {
        cudaFuncAttributes fa;
        M2_CUDA_TRY(cudaFuncGetAttributes(&fa, f));
        M2_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_optin - (int)fa.sharedSizeBytes));
    }
    for (const void* f : funcs) {
        cudaFuncAttributes fa;
        M2_CUDA_TRY(cudaFuncGetAttributes(&fa, f));
        M2_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_optin - (int)fa.sharedSizeBytes));
    }
    return M2_OK;
}

namespace {

// Work maps of a list of tasks (stage order per kernel class) and the workspace they need.
struct Maps {
    std::vector<int4> sp[3];
    std::vector<int4> co[6];
    size_t smem_cols[6] = {};
    std::vector<int4> ro;
    std::vector<int2> ep[3];  // by epilogue tile height 8, 16, 32
    std::vector<int2> epf;    // tasks with the F-statistic (16 x 16 tiles)
    int64_t ws_f2 = 0;  // workspace, float2 units
    size_t spread_smem_max = 16;  // largest shared memory a task's spread tiles need
    size_t spread_smem() const { return spread_smem_max; }
};

// Append task `task` of context c (geometry g) to the maps, in the CTA shapes of cfg; its
// workspace goes at the end.
void add_task(Maps& m, int task, const Ctx& c, int64_t ntiles, HTask& t, const HBConfig& cfg) {
    auto take = [&](int64_t n) {  // 256-byte aligned sections
        const int64_t o = m.ws_f2;
        m.ws_f2 += (n + 31) / 32 * 32;
        return o;
    };
    t.g_off = take((int64_t)c.Kp * c.Lg);
    t.z_off = take((int64_t)c.Kp * c.n1 * kRowLen);
    // spread: cfg.spread_tiles tiles per CTA
    const int kpc = c.Kp <= 2 ? 0 : (c.Kp <= 4 ? 1 : 2);
    const int nt = cfg.spread_tiles;
    m.spread_smem_max = std::max(m.spread_smem_max, packed::spread_ell_smem_bytes(c.Kp, 1, c.ecap, c.pcap, c.ncap));
    for (int64_t tile = 0; tile < ntiles; tile += nt)
        m.sp[kpc].push_back(make_int4(task, (int)tile, (int)std::min<int64_t>(nt, ntiles - tile), 0));
    // column DFTs: one coset per warp where the C = n1 / F cosets allow it (C = 1: four one-warp
    // groups per CTA, C = 2: two two-warp groups), else one four-warp group sharing the cosets
    const int C = c.n1 / c.F;
    const int gw = C == 1 ? 1 : (C == 2 ? 2 : 4);
    const int lf = packed::ilog2c(c.F);
    for (int j = 0; j < c.Kp; ++j)
        for (int col = 0; col < kRowLen; col += 32 * (4 / gw)) m.co[lf].push_back(make_int4(task, j, col, gw));
    m.smem_cols[lf] = std::max(m.smem_cols[lf], sizeof(float2) * (packed::cols_tw_f2(false, c.n1, c.rows, c.F) +
                                                                   (size_t)(4 / gw) * packed::cols_group_f2(false, c.rows, c.F, c.n1)));
    // row FFTs: up to cfg.row_warps rows per CTA
    const int rw = cfg.row_warps;
    for (int j = 0; j < c.Kp; ++j)
        for (int r0 = 0; r0 < c.n1; r0 += rw) m.ro.push_back(make_int4(task, j, r0, std::min(rw, c.n1 - r0)));
    // epilogue with the F-statistic: 16 x 16 tiles (every J_k of a position in one thread)
    if (t.F) {
        const int nf16 = packed::epi_tiles(c.n1, c.k2max, 16);
        for (int e = 0; e < nf16; ++e) m.epf.push_back(make_int2(task, e));
        return;
    }
    // epilogue: one T1 x 16 tile per CTA, T1 <= cfg.epi_t1 the height of 8, 16 or 32 rows that leaves
    // the fewest idle rows in the task's n1 rows (the largest on a tie): small signals (n1 = 6, 12, 24)
    // do not run 32-row tiles that are mostly empty
    int t1 = 8, best = -1;
    for (int cand : {8, 16, 32}) {
        if (cand > cfg.epi_t1) break;
        const int waste = (c.n1 + cand - 1) / cand * cand - c.n1;
        if (best < 0 || waste <= best) {
            best = waste;
            t1 = cand;
        }
    }
    const int cls = t1 == 8 ? 0 : (t1 == 16 ? 1 : 2);
    const int ntile = packed::epi_tiles(c.n1, c.k2max, t1);
    for (int e = 0; e < ntile; ++e) m.ep[cls].push_back(make_int2(task, e));
}

// Device work-map pointers and counts of one launch.
struct MapView {
    const int4* sp[3] = {};
    int n_sp[3] = {};
    size_t spread_smem = 0;  // dynamic shared memory of the spread launches
    const int4* co[6] = {};
    int n_co[6] = {};
    size_t smem_cols[6] = {};
    const int4* ro = nullptr;
    int n_ro = 0;
    const int2* ep[3] = {};
    int n_ep[3] = {};
    const int2* epf = nullptr;
    int n_epf = 0;
};

template <int NT>
void launch_spread_maps(const MapView& v, const HTask* tasks, const Ctx* ctxs, float2* ws, cudaStream_t st) {
    const size_t sm = v.spread_smem;
    if (v.n_sp[0]) hb_spread_kernel<2, NT><<<v.n_sp[0], kSpreadTile, sm, st>>>(v.sp[0], tasks, ctxs, ws);
    if (v.n_sp[1]) hb_spread_kernel<4, NT><<<v.n_sp[1], kSpreadTile, sm, st>>>(v.sp[1], tasks, ctxs, ws);
    if (v.n_sp[2]) hb_spread_kernel<8, NT><<<v.n_sp[2], kSpreadTile, sm, st>>>(v.sp[2], tasks, ctxs, ws);
}

m2_status launch_maps(const MapView& v, const HTask* tasks, const Ctx* ctxs, const Tw32& tw, float2* ws,
                      const HBConfig& cfg, cudaStream_t st) {
    if (cfg.spread_tiles == 1) launch_spread_maps<1>(v, tasks, ctxs, ws, st);
    else if (cfg.spread_tiles == 4) launch_spread_maps<4>(v, tasks, ctxs, ws, st);
    else launch_spread_maps<2>(v, tasks, ctxs, ws, st);
    M2_CUDA_TRY(cudaGetLastError());
    for (int k = 1; k < 6; ++k) {
        if (!v.n_co[k]) continue;
        const size_t sm = v.smem_cols[k];
        switch (k) {
            case 1: hb_cols_kernel<2><<<v.n_co[k], kColThreads, sm, st>>>(v.co[k], tasks, ctxs, tw, ws); break;
            case 2: hb_cols_kernel<4><<<v.n_co[k], kColThreads, sm, st>>>(v.co[k], tasks, ctxs, tw, ws); break;
            case 3: hb_cols_kernel<8><<<v.n_co[k], kColThreads, sm, st>>>(v.co[k], tasks, ctxs, tw, ws); break;
            case 4: hb_cols_kernel<16><<<v.n_co[k], kColThreads, sm, st>>>(v.co[k], tasks, ctxs, tw, ws); break;
            default: hb_cols_kernel<32><<<v.n_co[k], kColThreads, sm, st>>>(v.co[k], tasks, ctxs, tw, ws); break;
        }
        M2_CUDA_TRY(cudaGetLastError());
    }
    if (v.n_ro) {
        if (cfg.row_warps == 4)
            hb_rows_kernel<4><<<v.n_ro, 32 * 4, packed::rowfft_smem_bytes(4), st>>>(v.ro, tasks, ctxs, tw, ws);
        else hb_rows_kernel<8><<<v.n_ro, 32 * 8, packed::rowfft_smem_bytes(8), st>>>(v.ro, tasks, ctxs, tw, ws);
        M2_CUDA_TRY(cudaGetLastError());
    }
    if (v.n_epf) hb_epi_f_kernel<<<v.n_epf, 256, 0, st>>>(v.epf, tasks, ctxs, ws);
    if (v.n_ep[0]) hb_epi_kernel<8><<<v.n_ep[0], 16 * 8, 0, st>>>(v.ep[0], tasks, ctxs, ws);
    if (v.n_ep[1]) hb_epi_kernel<16><<<v.n_ep[1], 16 * 16, 0, st>>>(v.ep[1], tasks, ctxs, ws);
    if (v.n_ep[2]) hb_epi_kernel<32><<<v.n_ep[2], 16 * 32, 0, st>>>(v.ep[2], tasks, ctxs, ws);
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

}  // namespace

m2_status hbatch_create(m2nufft_plan_s* const* plans, const void* const* xs, int64_t nsig, void* const* Js,
                        void* const* Es, void* const* Ps, void* const* Fs, const HBConfig& cfg, HBatch** out) {
    if (!(cfg.spread_tiles == 1 || cfg.spread_tiles == 2 || cfg.spread_tiles == 4) ||
        !(cfg.row_warps == 4 || cfg.row_warps == 8) || !(cfg.epi_t1 == 16 || cfg.epi_t1 == 32)) {
        set_error("internal: unsupported stage-batched CTA shapes");
        return M2_ERR_ARG;
    }
    std::unique_ptr<HBatch> H(new HBatch());
    H->device = plans[0]->device;
    H->cfg = cfg;
    H->tw = packed::make_tw32();
    std::vector<Ctx> ctxs;
    std::map<const m2nufft_plan_s*, int> index;
    std::vector<HTask> tasks((size_t)nsig);
    Maps m;
    for (int64_t s = 0; s < nsig; ++s) {
        const m2nufft_plan_s* p = plans[s];
        auto f = index.find(p);
        if (f == index.end()) {
            f = index.emplace(p, (int)ctxs.size()).first;
            ctxs.push_back(packed_ctx(p));
        }
        HTask& t = tasks[(size_t)s];
        t.x = static_cast<const float*>(xs[s]);
        t.J = Js ? static_cast<float2*>(Js[s]) : nullptr;
        t.E = Es ? static_cast<float*>(Es[s]) : nullptr;
        t.P = Ps ? static_cast<float*>(Ps[s]) : nullptr;
        t.F = Fs ? static_cast<float*>(Fs[s]) : nullptr;
        t.ctx = f->second;
        t.pad0 = 0;
        add_task(m, (int)s, ctxs[(size_t)f->second], p->g.ntiles, t, cfg);
    }
    const int64_t off = m.ws_f2;
    std::vector<int4>* sp = m.sp;
    std::vector<int4>* co = m.co;
    std::vector<int4>& ro = m.ro;
    for (int k = 0; k < 6; ++k) H->smem_cols[k] = m.smem_cols[k];
    H->spread_smem = m.spread_smem();
    H->ws_bytes = (size_t)off * sizeof(float2);
    M2_CUDA_TRY(cudaMalloc(&H->ws, H->ws_bytes));
    H->owned.push_back(H->ws);
    M2_TRY(upload_vec(H->owned, &H->d_ctxs, ctxs));
    M2_TRY(upload_vec(H->owned, &H->d_tasks, tasks));
    for (int k = 0; k < 3; ++k) {
        M2_TRY(upload_vec(H->owned, &H->d_spread[k], sp[k]));
        H->n_spread[k] = (int)sp[k].size();
    }
    for (int k = 0; k < 6; ++k) {
        M2_TRY(upload_vec(H->owned, &H->d_cols[k], co[k]));
        H->n_cols[k] = (int)co[k].size();
    }
    M2_TRY(upload_vec(H->owned, &H->d_rows, ro));
    H->n_rows = (int)ro.size();
    for (int k = 0; k < 3; ++k) {
        M2_TRY(upload_vec(H->owned, &H->d_epi[k], m.ep[k]));
        H->n_epi[k] = (int)m.ep[k].size();
    }
    M2_TRY(upload_vec(H->owned, &H->d_epif, m.epf));
    H->n_epif = (int)m.epf.size();
    *out = H.release();
    return M2_OK;
}

// The batch's launches, in stage order, on one stream (captured into a graph by the caller).
m2_status hbatch_run(HBatch* H, cudaStream_t st) {
    MapView v;
    v.spread_smem = H->spread_smem;
    for (int k = 0; k < 3; ++k) {
        v.sp[k] = H->d_spread[k];
        v.n_sp[k] = H->n_spread[k];
    }
    for (int k = 0; k < 6; ++k) {
        v.co[k] = H->d_cols[k];
        v.n_co[k] = H->n_cols[k];
        v.smem_cols[k] = H->smem_cols[k];
    }
    v.ro = H->d_rows;
    v.n_ro = H->n_rows;
    for (int k = 0; k < 3; ++k) {
        v.ep[k] = H->d_epi[k];
        v.n_ep[k] = H->n_epi[k];
    }
    v.epf = H->d_epif;
    v.n_epf = H->n_epif;
    return launch_maps(v, H->d_tasks, H->d_ctxs, H->tw, H->ws, H->cfg, st);
}

int hbatch_launches(const HBatch* H) {
    int n = (H->n_rows ? 1 : 0) + (H->n_epif ? 1 : 0);
    for (int k = 0; k < 3; ++k) n += H->n_epi[k] ? 1 : 0;
    for (int k = 0; k < 3; ++k) n += H->n_spread[k] ? 1 : 0;
    for (int k = 0; k < 6; ++k) n += H->n_cols[k] ? 1 : 0;
    return n;
}

// ---------------------------------------------------------------------------
// Serving: the same stage kernels over the requests of one launch, whatever
// their sampling patterns.  The plan contexts stay on the device; each launch
// builds its task records and work maps on the host into a pinned staging
// buffer, copies them with one transfer and runs the stage launches.
// ---------------------------------------------------------------------------
struct HServe {
    std::vector<Ctx> ctxs;
    std::vector<int64_t> ntiles;
    Ctx* d_ctxs = nullptr;
    Tw32 tw;
    ~HServe() {
        if (d_ctxs) cudaFree(d_ctxs);
    }
};

m2_status hserve_create(m2nufft_plan_s* const* plans, int nplans, HServe** out) {
    std::unique_ptr<HServe> H(new HServe());
    H->tw = packed::make_tw32();
    for (int i = 0; i < nplans; ++i) {
        H->ctxs.push_back(packed_ctx(plans[i]));
        H->ntiles.push_back(plans[i]->g.ntiles);
    }
    M2_CUDA_TRY(cudaMalloc(&H->d_ctxs, sizeof(Ctx) * H->ctxs.size()));
    M2_CUDA_TRY(cudaMemcpy(H->d_ctxs, H->ctxs.data(), sizeof(Ctx) * H->ctxs.size(), cudaMemcpyHostToDevice));
    *out = H.release();
    return M2_OK;
}

void hserve_free(HServe* H) { delete H; }

size_t hserve_ws_bytes(const HServe* H, int plan) {
    Maps m;
    HTask t{};
    add_task(m, 0, H->ctxs[plan], H->ntiles[plan], t, HBConfig{});
    return sizeof(float2) * (size_t)m.ws_f2;
}

size_t hserve_map_bytes(const HServe* H, int plan) {
    Maps m;
    HTask t{};
    add_task(m, 0, H->ctxs[plan], H->ntiles[plan], t, HBConfig{});
    size_t b = sizeof(HTask);
    for (auto& v : m.sp) b += sizeof(int4) * v.size();
    for (auto& v : m.co) b += sizeof(int4) * v.size();
    b += sizeof(int4) * m.ro.size();
    for (auto& v : m.ep) b += sizeof(int2) * v.size();
    return b + 16 * 14;  // per-section alignment
}

m2_status hserve_launch(HServe* H, int n, const int* plan, const float* const* x, float2* const* J,
                        float* const* E, float* const* P, float2* ws, char* hstage, char* dstage, size_t stage_cap,
                        cudaStream_t st) {
    Maps m;
    std::vector<HTask> tasks((size_t)n);
    for (int r = 0; r < n; ++r) {
        HTask& t = tasks[(size_t)r];
        t.x = x[r];
        t.J = J ? J[r] : nullptr;
        t.E = E ? E[r] : nullptr;
        t.P = P[r];
        t.F = nullptr;
        t.ctx = plan[r];
        t.pad0 = 0;
        add_task(m, r, H->ctxs[plan[r]], H->ntiles[plan[r]], t, HBConfig{});
    }
    // staging layout: tasks, then the maps, each section 16-byte aligned
    size_t off = 0;
    auto put = [&](const void* src, size_t bytes) -> size_t {
        off = (off + 15) & ~size_t(15);
        const size_t o = off;
        if (bytes) std::memcpy(hstage + o, src, bytes);
        off += bytes;
        return o;
    };
    MapView v;
    const size_t ot = put(tasks.data(), sizeof(HTask) * tasks.size());
    size_t osp[3], oco[6];
    for (int k = 0; k < 3; ++k) osp[k] = put(m.sp[k].data(), sizeof(int4) * m.sp[k].size());
    for (int k = 0; k < 6; ++k) oco[k] = put(m.co[k].data(), sizeof(int4) * m.co[k].size());
    const size_t oro = put(m.ro.data(), sizeof(int4) * m.ro.size());
    size_t oep[3];
    for (int k = 0; k < 3; ++k) oep[k] = put(m.ep[k].data(), sizeof(int2) * m.ep[k].size());
    if (off > stage_cap) {
        set_error("internal: serving work maps (%zu bytes) exceed the staging buffer (%zu)", off, stage_cap);
        return M2_ERR_ARG;
    }
    M2_CUDA_TRY(cudaMemcpyAsync(dstage, hstage, off, cudaMemcpyHostToDevice, st));
    v.spread_smem = m.spread_smem();
    for (int k = 0; k < 3; ++k) {
        v.sp[k] = reinterpret_cast<const int4*>(dstage + osp[k]);
        v.n_sp[k] = (int)m.sp[k].size();
    }
    for (int k = 0; k < 6; ++k) {
        v.co[k] = reinterpret_cast<const int4*>(dstage + oco[k]);
        v.n_co[k] = (int)m.co[k].size();
        v.smem_cols[k] = m.smem_cols[k];
    }
    v.ro = reinterpret_cast<const int4*>(dstage + oro);
    v.n_ro = (int)m.ro.size();
    for (int k = 0; k < 3; ++k) {
        v.ep[k] = reinterpret_cast<const int2*>(dstage + oep[k]);
        v.n_ep[k] = (int)m.ep[k].size();
    }
    return launch_maps(v, reinterpret_cast<const HTask*>(dstage + ot), H->d_ctxs, H->tw, ws, HBConfig{}, st);
}

}  // namespace m2
