/*
 * m2serve.h -- native continuous-batching PSD server over cached M2NuFFT plans.
 *
 * The paper has no counterpart to this interface: it is the serving runtime
 * around the per-signal path of include/m2nufft.h.  Requests (pattern index,
 * host samples, arrival time) are admitted whenever a launch slot is free and
 * the request's device buffers fit that slot's share of the memory budget;
 * slots run on separate CUDA streams, so a new batch starts while earlier
 * batches are still on the GPU.  Latency = completion time (P-hat back in host
 * memory) minus arrival.
 *
 * Launches: when every plan is a packed FP32 plan (m2_info.path 2 or 3), a
 * launch takes up to max_batch queued requests of any patterns and runs them
 * through one set of stage launches (spread, column DFTs, row FFTs, epilogue
 * over all its requests, the work maps built per launch and copied with one
 * transfer, the workspace in the slot's arena): one H2D copy of the samples,
 * one D2H copy of the P-hats; a launch that holds a single request runs its
 * plan's own m2nufft_exec instead while that plan is in no other slot (no work
 * maps to stage).  Otherwise requests are grouped by pattern, each
 * group is one m2nufft_exec, and a pattern is in at most one slot at a time (a
 * plan's workspace serves one launch at a time).  Results do not depend on the
 * launch a request lands in.
 *
 * Memory: at create, each slot receives a device arena of
 * min((mem_budget - sum of plan device bytes) / slots, max_batch requests of the
 * largest pattern) bytes and a pinned host staging arena; nothing is allocated
 * while serving.
 */
#ifndef M2SERVE_H
#define M2SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "m2nufft.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct m2serve_s* m2serve_t;

/*
 * plans      host [nplans] FP32 plans (one per sampling pattern; not owned, must outlive the server)
 * mem_budget bytes of device memory for plans plus request buffers
 * slots      concurrent launch slots (CUDA streams), >= 1
 * max_batch  most requests per launch, >= 1
 * outputs    M2_OUT_J | M2_OUT_E | M2_OUT_P bits: device outputs computed per request (P always)
 * Errors: M2_ERR_ARG, M2_ERR_BUDGET (budget does not cover the plans plus one request
 * of the largest pattern per slot), M2_ERR_NOMEM, M2_ERR_CUDA.
 */
m2_status m2serve_create(const m2nufft_plan_t* plans, int nplans, size_t mem_budget, int slots, int max_batch,
                         unsigned outputs, m2serve_t* out);

/*
 * Replay a request trace in real time (arrival_s relative to the call).
 *   nreq       number of requests
 *   pattern    host [nreq] plan index of each request
 *   arrival_s  host [nreq] arrival times, seconds (need not be sorted)
 *   x          host [nreq] pointers to float32 samples [N of the pattern], in the order of t
 *   p_out      host [nreq] pointers receiving P-hat [I of the pattern] (float32), or NULL
 *   latency_s  host [nreq] output: completion minus arrival, seconds
 *   plain      0 = continuous batching; 1 = plain path (each request alone, B = 1,
 *              one stream, processed in arrival order as soon as it has arrived)
 * Synchronous; returns when every request has completed.
 */
m2_status m2serve_run_trace(m2serve_t s, int64_t nreq, const int32_t* pattern, const double* arrival_s,
                            const float* const* x, float* const* p_out, double* latency_s, int plain);

/* Number of launches and of requests served by the last run_trace. */
m2_status m2serve_stats(m2serve_t s, int64_t* launches, int64_t* requests);

m2_status m2serve_destroy(m2serve_t s);

#ifdef __cplusplus
}
#endif

#endif /* M2SERVE_H */
