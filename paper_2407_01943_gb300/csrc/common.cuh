// Shared definitions of the GB300 M2NuFFT library (plan + exec).
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "m2nufft.h"

namespace m2 {

void set_error(const char* fmt, ...);
void clear_error();

#define M2_CUDA_TRY(expr)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ::m2::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),        \
                            __FILE__, __LINE__);                                           \
            (void)cudaGetLastError(); /* reported here: not again by a later launch check */ \
            return e_ == cudaErrorMemoryAllocation ? M2_ERR_NOMEM : M2_ERR_CUDA;           \
        }                                                                                  \
    } while (0)

#define M2_TRY(expr)                      \
    do {                                  \
        m2_status s_ = (expr);            \
        if (s_ != M2_OK) return s_;       \
    } while (0)

template <typename R> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };

// Spreading tile: fine-grid cells per CTA of the spread kernel.
constexpr int kSpreadTile = 256;
// Points staged in shared memory per chunk of the spread kernel.
constexpr int kSpreadChunk = 256;
constexpr int kLanes = 2;  // packed path: consecutive chunks overlapped on this many internal streams
// Largest K the exec kernels are instantiated for.
constexpr int kMaxK = 16;

// Fine-grid / FFT geometry of one plan.
struct Geometry {
    int64_t N = 0;        // samples
    int K = 0;            // tapers
    int64_t I = 0;        // band centres
    double f_lo = 0, df = 0;
    int64_t i_c = 0;      // I / 2: band index of the mid frequency
    double fmid_hi = 0, fmid_lo = 0;  // f_lo + i_c df as a double-double
    int width = 0;        // spreading kernel width (cells)
    double beta = 0;      // ES kernel shape
    int64_t nf = 0;       // FFT length
    int log_nf = 0;
    int64_t n1 = 0, n2 = 0;  // nf = n1 * n2
    int log_n1 = 0, log_n2 = 0;
    int64_t rows = 0;     // nonzero rows of the column FFT input
    int64_t Lg = 0;       // spread-grid cells written per (signal, taper) = rows * n2
    int wrap = 0;         // support covers the whole period
    double h = 0;         // cell width in time units = 1 / (nf df)
    double t_ref = 0;     // time of fine-grid cell 0
    int real_taper = 1;   // modulated taper is real
    int64_t P = 0;        // number of (extended) spread points
    int64_t ntiles = 0;   // spread tiles
    int cw = 0;           // columns per CTA in the column pass
    int rw = 0;           // rows per CTA in the row pass
    int chunk = 1;        // signals per chunk
    int twb_bits = 0;     // low-bit width of the two-level nf twiddle table
    int path = 1;         // 1 = generic kernels, 2 = packed FP32 kernels, 3 = packed, persistent pipelined kernel
    int kp = 0;           // FFT signals per signal: K (generic) or ceil(K/2) taper pairs (packed)
    int colF = 0;         // packed path: coset FFT length F (largest power of two <= 32 dividing n1)
};

}  // namespace m2

struct m2nufft_plan_s;

namespace m2 {
// Instrumentation: records a CUDA event (begin = 0 / end = 1) around kernel `kernel`
// on stream `st` while timing is enabled for the plan.
void mark(m2nufft_plan_s* p, int kernel, int which, cudaStream_t st);
// Drop cached exec_batch graphs that reference plan p.
void purge_batch_graphs(const m2nufft_plan_s* p);
// One-time per-device set-up of the exec kernels' dynamic shared-memory limits.
m2_status init_exec_kernels(int smem_optin);
m2_status init_fast_kernels(int smem_optin);
m2_status init_pipe_kernels(int smem_optin);
m2_status init_device_kernels(int device);
// Sub-band nominal tapers (subband.cu): ts sorted; w_re, w_im [K][N], lam [K] descending.
m2_status solve_gep_subband(const std::vector<double>& ts, double f_w, int K, double f_c0, double f_min,
                            double f_max, size_t budget, std::vector<double>& w_re, std::vector<double>& w_im,
                            std::vector<double>& lam, double& seconds);
// Interpolated-DPSS nominal tapers (spline_tapers.cu): ts sorted; w_sorted [K][N], lam [K].
m2_status spline_tapers(const std::vector<double>& ts, double fmax, double fw, int K,
                        std::vector<double>& w_sorted, std::vector<double>& lam, double& seconds);
// M2_ERR_TIMEOUT (once) if a packed stage kernel of plan p gave up a bounded wait since the last check.
m2_status check_stage_status(m2nufft_plan_s* p);
// Packed FP32 path (fast.cu): one chunk of nb signals.
m2_status exec_fast_chunk(m2nufft_plan_s* p, const float* x, int nb, float2* J, float* E, float* P, float* F,
                          cudaStream_t st, int lane = 0, const float2* g_pre = nullptr);
// spread grids of nb signals (packed path) into g_out [nb][Kp][Lg]
m2_status spread_fast(m2nufft_plan_s* p, const float* x, int nb, float2* g_out, cudaStream_t st);
// Stage-batched executor of uneven batches of packed plans (hbatch.cu).  CTA shapes of its stage
// launches (every shape gives the same bits): spread tiles per CTA (1, 2, 4), row FFTs per CTA
// (4, 8), largest epilogue tile height T1 (16, 32; tiles T1 x 16, one position per thread; each task
// takes the height of 8, 16 or 32 up to it that leaves the fewest idle rows of its n1).  Tasks with
// an F-statistic output (Fs[s] non-NULL) take 16 x 16 epilogue tiles whatever the shape.
struct HBConfig {
    int spread_tiles = 2;
    int row_warps = 8;
    int epi_t1 = 32;
};
struct HBatch;
m2_status hbatch_create(m2nufft_plan_s* const* plans, const void* const* xs, int64_t nsig, void* const* Js,
                        void* const* Es, void* const* Ps, void* const* Fs, const HBConfig& cfg, HBatch** out);
m2_status hbatch_run(HBatch* H, cudaStream_t st);
int hbatch_launches(const HBatch* H);
void hbatch_free(HBatch* H);
m2_status init_hbatch_kernels(int smem_optin);
// Serving with the stage-batched kernels (hbatch.cu): plan contexts on the device, per-launch maps.
struct HServe;
m2_status hserve_create(m2nufft_plan_s* const* plans, int nplans, HServe** out);
void hserve_free(HServe* H);
size_t hserve_ws_bytes(const HServe* H, int plan);   // workspace of one request of that plan
size_t hserve_map_bytes(const HServe* H, int plan);  // staged task record and work maps of one request
m2_status hserve_launch(HServe* H, int n, const int* plan, const float* const* x, float2* const* J,
                        float* const* E, float* const* P, float2* ws, char* hstage, char* dstage, size_t stage_cap,
                        cudaStream_t st);
// Persistent pipelined kernel of the packed path (pipe.cu).
struct PipeLaunch;
void pipe_free(PipeLaunch* L);
// all B signals of plan p in one launch (cached launch configuration per B)
m2_status exec_pipe(m2nufft_plan_s* p, const float* x, int64_t B, float2* J, float* E, float* P, cudaStream_t st);
// create the cached launch configuration for B signals (not allowed during stream capture)
m2_status pipe_prepare(m2nufft_plan_s* p, int64_t B);
// uneven batch of packed plans: signal s of plans[s]; owns its ring workspace
m2_status pipe_batch_create(m2nufft_plan_s* const* plans, const void* const* xs, int64_t nsig, void* const* Js,
                            void* const* Es, void* const* Ps, PipeLaunch** out);
m2_status pipe_batch_run(PipeLaunch* L, cudaStream_t st);
// M2_ERR_TIMEOUT (once) if an earlier launch of L gave up waiting
m2_status pipe_check(PipeLaunch* L);
// a cached batch graph containing L was launched (its stage accounting is the one reported for NULL)
void pipe_batch_mark_launched(PipeLaunch* L);
// stage accounting of the most recently launched batch (device buffer of 12 counters), or NULL
unsigned long long* pipe_last_batch_profile(int* device);
}  // namespace m2

struct m2nufft_plan_s {
    m2::Geometry g;
    int device = 0;
    int sm_count = 0;  // multiprocessors of the device (grid sizing)
    int precision = 32;
    double fs = 1.0, f_w = 0.0;
    double tol = 0.0;
    int integer_grid = 0;
    int have_lambda = 0;
    int have_leakage = 0;
    double gep_seconds = 0.0;
    size_t device_bytes = 0;
    std::vector<double> t;       // caller order
    std::vector<double> w;       // [K][N] caller order (real part for sub-band plans)
    std::vector<double> w_im;    // [K][N] caller order, imaginary part (sub-band plans)
    int complex_taper = 0;       // sub-band plan: complex tapers, band grid relative to f_c0
    double f_c0 = 0.0;           // nominal band centre
    std::vector<double> lambda;  // [K] descending

    // device caches (precision-typed buffers are void*)
    int32_t* d_pt_src = nullptr;   // [P] index into x (caller order)
    int32_t* d_pt_cell = nullptr;  // [P] first fine-grid cell of the point's window
    void* d_pt_off = nullptr;      // [P] R: (first cell) - u_n, in cells
    void* d_taper = nullptr;       // [K][P] R (real taper) or C (modulated taper)
    int32_t* d_tile_pb = nullptr;  // [ntiles] first point of each spread tile
    int32_t* d_tile_pe = nullptr;  // [ntiles] one past the last point
    // packed path: cell-major spreading matrix (sliced ELL, 32-cell slices; the layout is described
    // at packed::spread_ell)
    int2* d_ell_slice = nullptr;  // per slice {first entry, entries per cell}
    uint2* d_ell_e = nullptr;     // per entry {point word, window value bits}
    int4* d_ell_tile = nullptr;   // per tile {first entry, entries, first point, points}
    int4* d_ell_run = nullptr;    // per tile {first sample, samples, staged, 0}
    float* d_tap2 = nullptr;      // [P][Kp] taper pairs, point-major (FP32 complex)
    int ell_ecap = 0, ell_pcap = 0, ell_ncap = 0;  // largest staged tile (multiples of 4)
    int64_t ell_entries = 0;      // entries including padding
    void* d_deconv = nullptr;      // [I] C: exp(-i 2 pi m df t_ref) / phihat(m)
    void* d_tw1 = nullptr;         // [n1/2] C: exp(-i 2 pi q / n1)
    void* d_tw2 = nullptr;         // [n2/2] C: exp(-i 2 pi q / n2)
    void* d_twa = nullptr;         // [nf >> twb_bits] C: exp(-i 2 pi (q << twb_bits) / nf)
    void* d_twb = nullptr;         // [1 << twb_bits]  C: exp(-i 2 pi q / nf)
    void* d_twn1 = nullptr;        // packed path: [n1] C, exp(-i 2 pi q / n1) full circle
    void* d_tw1024 = nullptr;      // packed path: [32][32] C, [cc][l] = exp(-i 2 pi cc l / 1024)
    void* d_colT = nullptr;        // packed path: [F][1024] C, exp(-i 2 pi l2 C q / nf) (column-FFT output twiddle)
    void* d_colB = nullptr;        // packed path: [C][1024] C, exp(-i 2 pi l2 r / nf) (per-coset factor)
    void* d_colFw = nullptr;       // packed path: [C][rows] C, exp(-i 2 pi ((l1 r) mod n1) / n1) (fold twiddles)
    void* d_wsum = nullptr;        // [K] R: W_k^0(0) = sum_n w_k(t_n) (F-statistic)
    double wq = 0.0;               // sum_k W_k^0(0)^2
    void* d_Jscratch = nullptr;    // generic path: J of one chunk when F is wanted without J
    double* d_Lhat = nullptr;      // [K][I]
    double* d_Ehat = nullptr;      // [I]
    void* d_g = nullptr;           // workspace [chunk][K][Lg] C
    void* d_Z = nullptr;           // workspace [chunk][K][nf] C (packed path: [chunk][K/2][n1][1024], the
                                   // column DFTs, then in place the in-band row transforms)
    // packed path, execs of more than one chunk: a second workspace and two internal streams, so
    // that chunk c's epilogue (HBM-bound) overlaps chunk c+1's spread and FFTs (issue-bound)
    void* d_gall = nullptr;  // packed path, multi-chunk execs: the spread grids of all signals
    int64_t gall_signals = 0;
    cudaEvent_t gall_ev = nullptr;  // recorded on the caller's stream after each exec that read d_gall
    void* lane_g[m2::kLanes] = {};  // lane L > 0 workspace (lane 0 uses d_g / d_Z)
    void* lane_Z[m2::kLanes] = {};
    cudaStream_t lane_st[m2::kLanes] = {};
    cudaEvent_t lane_ev[m2::kLanes] = {};
    cudaEvent_t fork_ev = nullptr;
    std::vector<void*> allocations;
    // persistent pipelined path: launch configurations by batch size, and a mapped pinned
    // status word [abort, status, item] that a launch writes if a wait gives up
    std::map<int64_t, m2::PipeLaunch*> pipe_cache;
    int* pipe_status = nullptr;
    // packed path: mapped pinned status word [flag, code, where, 0] that a stage kernel whose bounded
    // wait gave up writes (d_stage_status is its device address); exec reports it once
    int* stage_status = nullptr;
    int* d_stage_status = nullptr;
    // autotuning at plan time: the candidate configurations and their measured ms per exec
    std::vector<m2_opts> tune_opts;
    std::vector<double> tune_ms;
    unsigned long long* d_pipe_prof = nullptr;  // per-stage busy/wait accounting while timing is enabled

    // per-kernel timing (instrumentation): event pairs recorded by exec
    int timing = 0;
    std::vector<cudaEvent_t> ev_pool;       // free events
    std::vector<cudaEvent_t> ev_rec[4][2];  // [kernel][begin/end] in launch order
    double timing_ms[4] = {0, 0, 0, 0};
    int64_t timing_launches[4] = {0, 0, 0, 0};
};
