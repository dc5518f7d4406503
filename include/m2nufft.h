/*
 * m2nufft.h -- C ABI of the GB300 multitaper NuFFT power-spectrum path.
 *
 * Method: Cui, Brinkmann & Worrell, "Multiband-Multitaper Nonuniform FFT"
 * (arXiv 2407.01943).  Given samples x(t_n) at arbitrary times t_n
 * (n = 1..N), a signal band B = {|f| <= f_max} with f_max = fs/2, analysis
 * bands of half-width f_w and K tapers (Sec. 2; Table 1 steps 1-2), the
 * library
 *
 *   plan  : solves the nominal-band GEP R(A0) w = lambda R(B) w for the K
 *           largest eigenpairs in FP64 on the GPU (Sec. 3.2, Eq. gep_at_A0;
 *           Table 1 step 3), scales each taper to w^T R(B) w = 2 f_w
 *           (Sec. 2.2, Eq. bg_norm_requirement), and caches everything the
 *           per-signal path needs on the device;
 *   exec  : for every signal computes, for all I band centres
 *           f_i = f_lo + i*df (i = 0..I-1), the eigencoefficients
 *               J_k(A_i) = sum_n w_k(t_n) x(t_n) exp(-i 2 pi f_i t_n)
 *           (Sec. 3.2, Eq. eigencoefficients; Table 1 step 4), the
 *           eigenspectra |J_k(A_i)|^2 and the estimate
 *               P(A_i) = (1/K) sum_k |J_k(A_i)|^2
 *           (Eq. power_spectrum_estimator; Table 1 step 5), and hands out
 *           the suboptimality estimates L_k^i = |lambda_k - lambda_hat_k^i|
 *           and E_i = (1/K) sum_k L_k^i (Sec. 3.5; App. B, Eq. lambda_hat_ki).
 *
 * The nominal band is centred at f_c0 = 0, so the frequency shift of
 * Eq. (freq_shift_op) is the band centre itself and the tapers are real.
 * The sum over n is evaluated by a nonuniform FFT to a relative accuracy set
 * by m2_opts.tol; the sum itself is exact by definition.
 *
 * Conventions for every call:
 *   - Pointers documented as "host" are read or written synchronously.
 *     Pointers documented as "device" must be CUDA device (or managed)
 *     memory of the plan's device.
 *   - The caller owns every buffer it passes.  A plan copies what it needs
 *     from t and owns all its device caches until m2nufft_destroy.
 *   - Real arrays have the plan's precision: float for precision 32, double
 *     for precision 64.  Complex arrays are interleaved (re, im) pairs of
 *     that type.  L-hat and E-hat are always double.
 *   - Every call returns an m2_status; on failure m2nufft_last_error()
 *     returns a message for the calling thread.  No call aborts the process
 *     and no C++ exception crosses this interface.
 */
#ifndef M2NUFFT_H
#define M2NUFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct m2nufft_plan_s* m2nufft_plan_t;

typedef enum {
    M2_OK = 0,
    M2_ERR_ARG = 1,        /* invalid argument (sizes, NaN/inf times, f_w outside (0, fs/2), ...) */
    M2_ERR_NOMEM = 2,      /* device or host allocation failed */
    M2_ERR_BUDGET = 3,     /* the plan would exceed m2_opts.mem_budget */
    M2_ERR_GEP = 4,        /* GEP failed (e.g. R(B) not positive definite in FP64: repeated times) */
    M2_ERR_CUDA = 5,       /* a CUDA runtime / library call failed */
    M2_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up */
    M2_ERR_CANCELLED = 7   /* work was cancelled by the caller */
} m2_status;

/* Band centres f_i = f_lo + i*df, i = 0..I-1 (Sec. 3.1: identical analysis
 * bands that differ only by a frequency shift).  Requires df > 0, I >= 1. */
typedef struct {
    double f_lo;
    double df;
    int64_t I;
} m2_fgrid;

/* Sub-band of the multiband partition (Sec. 2.3 and Sec. 3): the signal band
 * restricted to f_min <= |f| <= f_max, with the nominal analysis band
 * |f - f_c0| <= f_w inside it.  f_min = 0, f_max = fs/2, f_c0 = 0 is the full
 * band of m2nufft_plan. */
typedef struct {
    double f_c0;   /* nominal band centre */
    double f_min;  /* 0 <= f_min < f_max */
    double f_max;  /* <= fs/2 */
} m2_subband;

/* Output selection bits (informational; exec writes whatever pointers are non-NULL). */
enum {
    M2_OUT_J = 1,
    M2_OUT_E = 2,
    M2_OUT_P = 4,
    M2_OUT_LHAT = 8,
    M2_OUT_EHAT = 16
};

typedef struct {
    int precision;      /* 32 (FP32 spread/FFT, FP64-split coordinates) or 64 */
    double tol;         /* target relative accuracy of the NuFFT; <= 0 selects
                           1e-6 for precision 32 and 1e-12 for precision 64 */
    size_t mem_budget;  /* maximum bytes of device memory the plan may hold
                           (including GEP scratch); 0 = unlimited */
    int device;         /* CUDA device ordinal; < 0 = the caller's current device */
    int max_batch;      /* signals per internal chunk; <= 0 = automatic.  Packed paths: the chunk
                           (at most 64); generic path: an upper bound on the automatic chunk */
    int path;           /* exec kernels: 0 = automatic (2 where the plan qualifies, else 1),
                           1 = generic (any precision/grid),
                           2 = packed FP32 path as four kernels per chunk of signals,
                           3 = packed FP32 path as one persistent pipelined kernel per exec;
                           2 and 3 need real tapers, nf >= 2048 and a support of <= 64 rows
                           of 1024 cells (M2_ERR_ARG if the plan does not qualify) */
    int tapers;         /* m2nufft_plan only: 0 = GEP (Eq. gep_at_A0, dense FP64, O(N^3)),
                           1 = interpolated DPSS (Table 1 step 3 a-c: DPSS on N uniform nodes
                           from t_1 to t_N, not-a-knot cubic spline to t, scaled to
                           w^T R(B) w = 2 f_w; O(N) host work plus an O(N^2) FP64 pair sum on
                           the GPU; eigenvalues = the concentrations w^T R(A0) w / w^T R(B) w) */
    double sigma;       /* minimum oversampling nf / I: 0 = automatic (1.5 on the packed path with
                           the width ceil(1.25 log10(1/tol)) + 1; 2 on the generic path); at 2 or
                           more the width is ceil(log10(1/tol)) + 1; packed plans below 1.5 (nf
                           may then be 5 * 2^a) take ceil(ln(1/tol) / (pi sqrt(1 - 1/sigma))) + 1;
                           accepted range [1.25, 8] */
    int tune;           /* 1 = autotune at plan time (m2nufft_plan / _with_tapers, packed FP32 plans):
                           candidate configurations -- sigma 1.5 or 2, 4, 8 or 16 signals per
                           chunk, the four-kernel or the persistent path -- are built from the
                           same tapers and timed on a synthetic batch of 32 signals on the device; the fastest is kept (m2nufft_get_tuning reports them) */
} m2_opts;

/* Geometry of a plan, for callers that size buffers or compute rooflines. */
typedef struct {
    int64_t N;           /* number of samples */
    int K;               /* tapers */
    int64_t I;           /* band centres */
    int precision;       /* 32 or 64 */
    int width;           /* spreading kernel width in fine-grid cells */
    double beta;         /* exponential-of-semicircle kernel shape */
    int64_t nf;          /* fine-grid (FFT) length, a power of two >= 2 I */
    int64_t n1, n2;      /* nf = n1 * n2: column-FFT and row-FFT lengths */
    int64_t rows;        /* nonzero input rows of the column FFTs (support / n2) */
    int wrap;            /* 1 when the sampling span covers a whole 1/df period */
    int real_taper;      /* 1 when the modulated tapers are real (f_lo + (I/2) df == 0) */
    int integer_grid;    /* 1 when fs * t_n are all integers, so R(B) = I */
    int chunk;           /* signals per internal chunk */
    int path;            /* exec kernels in use: 1 = generic, 2 = packed FP32 (four kernels),
                            3 = packed FP32 (persistent pipelined kernel) */
    size_t device_bytes; /* device memory held by the plan */
    double gep_seconds;  /* wall time of the GEP during planning (0 if tapers were given) */
    int64_t spread_entries; /* packed paths: entries of the cell-major spreading matrix (each a
                               sample index and ceil(K/2) complex FP32 weights), padding
                               included; 0 on the generic path */
} m2_info;

/*
 * Create a plan for sampling times t and band-centre grid fc.
 *   t      host, length N, any order (no sorting required); FP64
 *   N      number of samples, >= 1
 *   fs     nominal sampling rate; the signal band is |f| <= fs/2 (Sec. 2;
 *          f_max = 1/2 for unit-rate data, Sec. 4)
 *   f_w    half-bandwidth of every analysis band, 0 < f_w < fs/2
 *   K      number of tapers, 1 <= K <= min(N, 16)
 *   fc     host, band-centre grid
 *   opts   host, may be NULL for defaults (precision 32)
 *   out    host, receives the plan handle
 * Solves the GEP with cuSOLVER in FP64 (dense, O(N^3)); synchronous.
 * Errors: M2_ERR_ARG, M2_ERR_GEP, M2_ERR_NOMEM, M2_ERR_BUDGET, M2_ERR_CUDA.
 */
m2_status m2nufft_plan(const double* t, int64_t N, double fs, double f_w, int K,
                       const m2_fgrid* fc, const m2_opts* opts, m2nufft_plan_t* out);

/*
 * Same as m2nufft_plan but with caller-supplied tapers instead of the GEP
 * (for tapers designed elsewhere, e.g. interpolated DPSS, Table 1 step 3a-c).
 *   w       host [K][N] FP64, in the order of t
 *   lambda  host [K] FP64 eigenvalues used by L-hat/E-hat, or NULL (then
 *           exec rejects requests for L-hat and E-hat)
 * Repeated times are allowed here.
 */
m2_status m2nufft_plan_with_tapers(const double* t, int64_t N, double fs, double f_w, int K,
                                   const m2_fgrid* fc, const double* w, const double* lambda,
                                   const m2_opts* opts, m2nufft_plan_t* out);

/*
 * Plan for one sub-band of a multiband partition (Q > 1; Sec. 2.3, Sec. 3,
 * Table 1 steps 2-4 per sub-band q).  The nominal tapers solve Eq. gep_at_A0
 * with R(A0) centred at f_c0 (complex Hermitian, Eq. gpss_matrix_a) against the
 * sub-band matrix R(B^q) (Eq. gpss_matrix_b_q), normalised to
 * w^H R(B^q) w = 2 f_w; the eigencoefficients of the band centred at f_ci are
 *   J_k(A_i) = sum_n conj(w_k(t_n)) x(t_n) e^{-i 2 pi (f_ci - f_c0) t_n}
 * (Eq. eigencoefficients with Delta f_i = f_ci - f_c0), and P-hat as usual.
 *   sb      host, the sub-band and nominal centre
 *   fc      host, the absolute band centres f_ci = f_lo + i df of this sub-band
 *   w       host [K][N] complex (re, im interleaved) tapers in the order of t, or
 *           NULL to solve the GEP (FP64, cuSOLVER).  R(B^q) is numerically
 *           singular once N exceeds 2 (f_max - f_min) T, so the GEP is solved on
 *           its numerical range (eigenvalues above 1e-9 of the largest): a
 *           standard Hermitian eigenproblem of the reduced matrix
 *   lambda  host [K] eigenvalues when w is given, or NULL
 * The tapers are complex, so exec runs the generic path (either precision);
 * the F-statistic is not formed for sub-band plans.  The leakage estimates
 * (App. B, taken with R(B^q) and the shifts f_ci - f_c0 from the nominal
 * centre) are formed by the direct FP64 pair sum when the eigenvalues are known
 * and N^2 I <= 1e9; otherwise exec rejects requests for them.
 * The phase of each taper is fixed by making
 * sum_n w_k(t_n) e^{-i 2 pi f_c0 t_n} (t_n - tbar)^(k mod 2) real and positive.
 * A multiband analysis is Q such plans (one per sub-band) run on the same x,
 * e.g. with one m2nufft_exec_batch call.
 * Errors: as m2nufft_plan; M2_ERR_ARG when the nominal band is not inside the
 * sub-band; M2_ERR_GEP when K exceeds the numerical rank of R(B^q).
 */
m2_status m2nufft_plan_subband(const double* t, int64_t N, double fs, double f_w, int K, const m2_subband* sb,
                               const m2_fgrid* fc, const double* w, const double* lambda, const m2_opts* opts,
                               m2nufft_plan_t* out);

/*
 * Run the per-signal path for B signals that share the plan's sampling times.
 * Output buffers (J, E, P, Lhat, Ehat here and in every exec entry point) may be
 * device memory or page-locked host memory that the device addresses directly
 * (cudaHostAlloc, or pinned memory under unified addressing): the kernels then
 * write the results straight into host memory over the host link, with no
 * separate copy.
 *   x      device [B][N] real (plan precision), each row in the order of t
 *   B      number of signals, >= 0 (0 is a no-op)
 *   J      device [B][K][I] complex, or NULL
 *   E      device [B][K][I] real eigenspectra |J|^2, or NULL
 *   P      device [B][I] real multitaper estimate, or NULL
 *   Lhat   device [K][I] double leakage estimates L_k^i, or NULL
 *   Ehat   device [I] double taper-averaged leakage E_i, or NULL
 *   stream cudaStream_t to enqueue on (NULL = legacy default stream)
 * Asynchronous: returns once the work is enqueued.  Launch errors are
 * reported here; device faults surface at the caller's next synchronisation.
 * Calls on one plan must not overlap on the device (they share the plan's
 * workspace); order them on one stream or synchronise between streams.
 * Path 2 with B above the plan's chunk: the spread grids of all B signals are
 * made in one launch first (kept by the plan, B * ceil(K/2) * rows * 1024
 * complex, up to 256 MiB; larger batches spread per chunk), then the chunks run
 * alternately on two internal streams with a second chunk workspace, forked
 * from and joined back to `stream`.  Both buffers are allocated on first use
 * (the grid buffer grows with B: before freeing the old one, the call waits on
 * the host for this plan's last exec that read it), so the first such call, and
 * a call that grows the buffer, is not capturable into a CUDA graph.
 * Path 3 runs all B signals in one launch; the first call for a new B builds
 * that launch's work list (synchronous upload, not allowed during stream
 * capture).  Its inter-CTA waits are bounded (2 s each): a launch that gave up
 * writes a status word, and the next exec on the plan returns M2_ERR_TIMEOUT.
 */
m2_status m2nufft_exec(m2nufft_plan_t p, const void* x, int64_t B, void* J, void* E, void* P,
                       double* Lhat, double* Ehat, void* stream);

/*
 * As m2nufft_exec, plus Thomson's F-statistic for a spectral line at every
 * band centre (Sec. 3, Eq. f_stat and the amplitude estimate after it):
 *   C_i = sum_k J_k(A_i) W_k / sum_k W_k^2,   W_k = W_k^0(0) = sum_n w_k(t_n),
 *   F_i = |C_i|^2 (K - 1) sum_k W_k^2 / sum_k |J_k(A_i) - C_i W_k|^2,
 * distributed F(2, 2K - 2) under the no-line hypothesis (bands with
 * 2 f_i > f_w).  W_k is formed in FP64 at plan time.
 *   F      device [B][I] real (plan precision), required
 *   J,E,P  as for m2nufft_exec, each may be NULL
 * The packed path (2 or 3) forms F in its epilogue from the eigencoefficients
 * it already holds (a path-3 plan runs its four-kernel form for this call);
 * the generic path runs one more kernel over J (an internal J buffer of one
 * chunk is allocated on first use when J is NULL).
 * Errors: as m2nufft_exec; M2_ERR_ARG for K < 2 or F == NULL.
 */
m2_status m2nufft_exec_ftest(m2nufft_plan_t p, const void* x, int64_t B, void* J, void* E, void* P, void* F,
                             void* stream);

/*
 * Uneven batch: nsig signals, each with its own plan (plans may repeat).
 *   plans  host [nsig] plan handles
 *   xs     host [nsig] device pointers, xs[s] -> [N_s] real
 *   Js, Es, Ps  host [nsig] device pointers ([K_s][I_s] complex, [K_s][I_s]
 *          real, [I_s] real); an entry or a whole array may be NULL
 *   stream as for m2nufft_exec
 * All plans must share one precision and one device.  The whole batch runs
 * as one CUDA graph launched on `stream`, cached per (plans, buffer pointers,
 * batch mode) and replayed on later calls with the same arguments (the first
 * call for a new set of arguments builds and instantiates it).  When every
 * plan is a packed FP32 plan (path 2 or 3) the graph holds, in batch mode 0
 * (default), one launch per stage over all nsig signals (spread, column DFTs
 * per coset length, row FFTs, epilogue) with a workspace for every signal, or,
 * in batch mode 1, a single launch of the persistent pipelined kernel with a
 * workspace ring, or, in batch mode 2, whichever of those forms measured
 * fastest for this batch (see m2nufft_set_batch_mode); the plans' own
 * workspaces are not used.  Otherwise signals
 * of different plans run concurrently on internal streams inside the graph
 * (signals of one plan in order).  Results are bit-identical to m2nufft_exec
 * on each signal's plan.  A plan in the batch must not be used by other work
 * that overlaps the batch on the device.  M2_ERR_TIMEOUT: an earlier replay
 * of this batch gave up a bounded wait (batch mode 1; see m2nufft_exec).
 */
m2_status m2nufft_exec_batch(const m2nufft_plan_t* plans, const void* const* xs, int64_t nsig,
                             void* const* Js, void* const* Es, void* const* Ps, void* stream);

/*
 * As m2nufft_exec_batch, plus Thomson's F-statistic (Sec. 3, Eq. f_stat; the
 * definition as for m2nufft_exec_ftest) for the signals that ask for it:
 *   Fs     host [nsig] device pointers, Fs[s] -> [I_s] real, or NULL entries
 *          (no F for that signal); the array itself is required
 * Every signal with an F output needs a full-band plan (real tapers) with
 * K >= 2.  All-packed batches run stage-batched in batch modes 0 and 1 (the
 * persistent kernel forms no F; its tasks take the 16 x 16 epilogue tiles of
 * the four-kernel path); batch mode 2 tunes over the stage-batched shapes
 * only.  Results are bit-identical to m2nufft_exec_ftest on each signal's
 * plan.  The graph cache key includes the F pointers.
 * Errors: as m2nufft_exec_batch; M2_ERR_ARG for Fs == NULL, or for a signal
 * with an F output whose plan has K < 2 or complex (sub-band) tapers.
 */
m2_status m2nufft_exec_batch_ftest(const m2nufft_plan_t* plans, const void* const* xs, int64_t nsig,
                                   void* const* Js, void* const* Es, void* const* Ps, void* const* Fs,
                                   void* stream);

/* Select how m2nufft_exec_batch runs all-packed batches (process-wide):
 * 0 = one launch per stage (default; spread 2 tiles per CTA, row FFTs 8 rows
 * per CTA, epilogue tiles of 32 x 16 positions), 1 = one persistent pipelined
 * kernel, 2 = autotuned: the first call for a batch (same plans and buffers)
 * builds every candidate -- the stage-per-launch form with spread tiles per CTA
 * 1, 2 or 4, rows per CTA 8 or 4 and epilogue tiles 32 x 16 or 16 x 16, and the
 * persistent kernel -- times each on `stream` (one warm-up launch, then the
 * mean of three; the batch's outputs are written each time, with the same bits
 * whichever candidate runs) and caches the fastest; later calls replay it.
 * That first call synchronises and cannot be captured (M2_ERR_ARG while
 * `stream` is capturing).  Returns the previous mode, or -1 for an invalid
 * mode. */
int m2nufft_set_batch_mode(int mode);

/* Report of the most recent batch tuned in batch mode 2: *n (in: capacity of
 * the arrays, out: number of candidates timed, 13 for all-packed batches),
 * config host [*n][4] or NULL: (batch mode 0 or 1, spread tiles per CTA,
 * rows per CTA, epilogue tile height) of each candidate, and ms host [*n] or
 * NULL: its measured milliseconds per batch.  The fastest is the one cached.
 * No counterpart in the paper (an autotuning report).  Errors: M2_ERR_ARG for
 * n == NULL or *n < 0. */
m2_status m2nufft_get_batch_tuning(int* n, int* config, double* ms);

/* Autotuning report of a plan made with m2_opts.tune = 1: *n candidate configurations (0 for
 * an untuned plan), their options (host [*n] or NULL; path 2/3, sigma, max_batch as tried) and the
 * measured ms per exec of a synthetic batch of 32 signals (host [*n] or NULL; 1e300 for
 * a candidate the plan does not admit).  Call with NULL arrays first to get *n (at most 8). */
m2_status m2nufft_get_tuning(m2nufft_plan_t p, int* n, m2_opts* opts, double* ms);

/* Copy the plan's tapers (host [K][N] FP64, order of t) and eigenvalues
 * (host [K], descending; NaN when the plan was made from caller tapers
 * without eigenvalues).  Either pointer may be NULL. */
m2_status m2nufft_get_tapers(m2nufft_plan_t p, double* w, double* lambda);

/* Complex tapers (host [K][N], re and im interleaved, order of t) and eigenvalues (host [K]); for a
 * full-band plan the imaginary parts are 0.  m2nufft_get_tapers rejects sub-band plans. */
m2_status m2nufft_get_tapers_complex(m2nufft_plan_t p, double* w, double* lambda);

/* Copy L-hat (host [K][I]) and E-hat (host [I]); either may be NULL. */
m2_status m2nufft_get_leakage(m2nufft_plan_t p, double* Lhat, double* Ehat);

/* Fill *info with the plan's geometry. */
m2_status m2nufft_get_info(m2nufft_plan_t p, m2_info* info);

/*
 * Instrumentation (no counterpart in the paper): per-kernel device timing.
 * While enabled, exec records a CUDA event pair around every kernel launch on
 * the launching stream.  m2nufft_get_timing waits for those events, returns
 * the summed milliseconds and launch counts of the exec kernels accumulated
 * since the previous call (index 0 = spread, 1 = column FFT, 2 = row FFT,
 * 3 = separate epilogue of the packed path; the generic path fuses its
 * epilogue into index 2; path 3 records its single persistent kernel at
 * index 0), and resets the accumulators.
 *   ms        host [4] or NULL
 *   launches  host [4] or NULL
 */
m2_status m2nufft_set_timing(m2nufft_plan_t p, int enable);
m2_status m2nufft_get_timing(m2nufft_plan_t p, double* ms, int64_t* launches);

/*
 * Instrumentation of the persistent pipelined kernel: each work item adds
 * its duration (after its dependency wait), and the time spent waiting for
 * that dependency, to per-stage sums.  For a plan p (path 3) the sums cover
 * its exec launches made while timing was enabled (m2nufft_set_timing); for
 * p = NULL they cover the launches of the most recently launched
 * all-packed m2nufft_exec_batch graph.  Returns the sums since the previous
 * call and resets them; synchronises the device.  Index 0 = spread,
 * 1 = column DFTs, 2 = row FFTs, 3 = epilogue.  Durations are summed over
 * work items (CTA time, not wall time): their ratios give the stage split.
 *   busy_ms, wait_ms  host [4] or NULL;  items  host [4] or NULL
 */
m2_status m2nufft_get_pipe_profile(m2nufft_plan_t p, double* busy_ms, double* wait_ms, int64_t* items);

/*
 * Leakage estimate without a plan and without allocating.  The paper has no
 * counterpart to this entry point: it computes the same L-hat / E-hat as
 * m2nufft_get_leakage returns for a plan with these tapers and eigenvalues,
 * by the direct pair sum.
 *
 * For callers that may not call cudaMalloc: code running where the device
 * allocator is off limits, e.g. worker threads of a host that reserves all
 * device memory at start-up and hands out buffers from its own pool, or
 * latency-critical loops where an allocation could synchronise the device
 * and stall other work.  Such callers cannot create a plan (planning
 * allocates), so everything here is passed in: the caller's own device
 * buffers for inputs and outputs, plus a fixed 32 MiB scratch array that is
 * part of this library's device image (every GPU that loads the library holds
 * it until the process exits).  No cudaMalloc, cudaFree or allocating
 * library routine is called.
 *
 *   t       device [N] FP64 sampling times (any order)
 *   N       1 <= N <= 2^20
 *   fs,f_w  as for m2nufft_plan (signal band |f| <= fs/2, 0 < f_w < fs/2)
 *   K       1 <= K <= 16
 *   fc      host, band-centre grid f_i = f_lo + i df, i < I
 *   w       device [K][N] FP64 tapers in the order of t
 *   lambda  device [K] FP64 nominal eigenvalues
 *   Lhat    device [K][I] FP64 output, L_k^i = |lambda_k - lambda_k 2 f_w / D_k^i|
 *   Ehat    device [I] FP64 output, E_i = (1/K) sum_k L_k^i
 *   stream  cudaStream_t (NULL = legacy default stream); asynchronous
 * Work is O(N^2 I K).  The scratch holds ceil(N/64) partial sums of K x I
 * doubles: calls needing more than 32 MiB return M2_ERR_ARG with a message.
 * Each call made outside stream capture looks up the scratch array's device
 * address on the current device (cudaGetSymbolAddress); a call on a capturing
 * stream uses the address found by the last call on that device outside
 * capture, so the first call on a device must come before any stream capture
 * (otherwise M2_ERR_ARG), and a capture made after cudaDeviceReset needs one
 * uncaptured call first.  All calls share the one array, which keeps the last
 * call's partial sums (each call writes every entry it later reads), so calls
 * that overlap on the GPU race: order them on one stream.
 */
m2_status m2nufft_leakage_static(const double* t, int64_t N, double fs, double f_w, int K,
                                 const m2_fgrid* fc, const double* w, const double* lambda,
                                 double* Lhat, double* Ehat, void* stream);

/*
 * Self-test of the bounded waits of the persistent pipelined kernel (no
 * counterpart in the paper).  Launches that kernel on one work item whose
 * dependency counter is never incremented, waits for it on `stream`, and
 * returns M2_ERR_TIMEOUT when the wait gave up after timeout_ms (1..10000),
 * the kernel returned and its status word names work item 0 -- the expected
 * outcome; any other outcome returns M2_ERR_CUDA.  Faults and hangs nothing:
 * the wait is bounded by the device's global timer.  Synchronous.
 */
m2_status m2nufft_pipe_selftest(int timeout_ms, void* stream);

/*
 * The suboptimality measure with the optimal per-band eigenvalues (Sec. 3,
 * Eq. subopt_measure):  E_i = (1/K) sum_k |lambda_k^i - lambda_k^0|, where
 * lambda_k^i are the K largest eigenvalues of the GEP at band A_i itself,
 * R(A_i) w = lambda R(B) w (R(A_i) = Eq. gpss_matrix_a centred at f_i), and
 * lambda_k^0 the plan's nominal eigenvalues.  It is what L-hat / E-hat estimate
 * without per-band GEPs; this entry point computes it exactly for small
 * problems (FP64 on the GPU: one Cholesky of R(B), batched reductions, one
 * Hermitian eigenvalue solve per band).  Synchronous.
 *   E         host [I] output
 *   lam_band  host [I][K] output (per-band eigenvalues, descending) or NULL
 * Errors: M2_ERR_ARG for sub-band plans, plans without eigenvalues, or
 * N > 512 or I N^3 > 4e12; M2_ERR_GEP when R(B) is not positive definite.
 */
m2_status m2nufft_true_suboptimality(m2nufft_plan_t p, double* E, double* lam_band);

/* Release every resource of the plan (synchronises its device first).  NULL is a no-op. */
m2_status m2nufft_destroy(m2nufft_plan_t p);

/* Message describing the calling thread's most recent failure ("" if none). */
const char* m2nufft_last_error(void);

/* Library version string. */
const char* m2nufft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* M2NUFFT_H */
