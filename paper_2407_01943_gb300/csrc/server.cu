// Native continuous-batching PSD server (include/m2serve.h).
//
// Host-side runtime: real-time trace replay, admission into launch slots (CUDA
// streams) with per-slot device and pinned-host arenas carved at create time,
// and completion by event polling.  When every plan is a packed FP32 plan, a
// launch runs all its requests, whatever their sampling patterns, through the
// stage-batched kernels (one set of stage launches over the launch's requests,
// work maps built per launch, workspace in the slot's arena) -- except a launch of
// a single request, which runs its plan's own exec when that plan is not in use in
// another slot; otherwise the requests are grouped by pattern and each group is one
// m2nufft_exec.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "common.cuh"
#include "m2serve.h"

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

struct Group {
    int pattern = 0;
    std::vector<int64_t> reqs;
    size_t dx = 0, dJ = 0, dE = 0, dP = 0;  // device arena offsets
    size_t hx = 0, hP = 0;                  // pinned arena offsets
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    char* dev = nullptr;
    size_t dev_cap = 0;
    char* host = nullptr;
    size_t host_cap = 0;
    bool busy = false;
    std::vector<Group> groups;
    // cross-pattern launches: the requests and the pinned offsets of their P-hat
    std::vector<std::pair<int64_t, size_t>> cross;
};

struct PlanGeo {
    int64_t N = 0, I = 0;
    int K = 0;
};

}  // namespace

struct m2serve_s {
    int device = 0;
    std::vector<m2nufft_plan_t> plans;
    std::vector<PlanGeo> geo;
    unsigned outputs = M2_OUT_P;
    int max_batch = 1;
    std::vector<Slot> slots;
    int64_t last_launches = 0, last_requests = 0;
    m2::HServe* hs = nullptr;                // cross-pattern launches (all plans packed), else NULL
    std::vector<size_t> ws_bytes, map_bytes;  // per request of each plan (cross-pattern launches)
};

namespace {

struct DevGuard {
    int prev = -1;
    bool changed = false;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DevGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

size_t dev_bytes(const m2serve_s* s, int pat, int64_t B) {
    const PlanGeo& g = s->geo[pat];
    size_t b = align_up(sizeof(float) * B * g.N) + align_up(sizeof(float) * B * g.I);
    if (s->outputs & M2_OUT_J) b += align_up(sizeof(float2) * B * g.K * g.I);
    if (s->outputs & M2_OUT_E) b += align_up(sizeof(float) * B * g.K * g.I);
    return b;
}
size_t host_bytes(const m2serve_s* s, int pat, int64_t B) {
    const PlanGeo& g = s->geo[pat];
    return align_up(sizeof(float) * B * g.N) + align_up(sizeof(float) * B * g.I);
}
// one request in a cross-pattern launch: its buffers, workspace and staged work maps
size_t cross_dev_bytes(const m2serve_s* s, int pat) {
    return dev_bytes(s, pat, 1) + align_up(s->ws_bytes[pat]) + align_up(s->map_bytes[pat]);
}
size_t cross_host_bytes(const m2serve_s* s, int pat) { return host_bytes(s, pat, 1) + align_up(s->map_bytes[pat]); }

void destroy_server(m2serve_s* s) {
    if (!s) return;
    {
        DevGuard guard(s->device);
        if (s->hs) m2::hserve_free(s->hs);
        for (Slot& sl : s->slots) {
            if (sl.stream) cudaStreamSynchronize(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.stream) cudaStreamDestroy(sl.stream);
            cudaFree(sl.dev);
            cudaFreeHost(sl.host);
        }
    }
    delete s;
}

using Clock = std::chrono::steady_clock;

struct Run {
    m2serve_s* s;
    int64_t nreq;
    const int32_t* pattern;
    const double* arrival;
    const float* const* x;
    float* const* p_out;
    double* latency;
    Clock::time_point t0;
    std::vector<int> pattern_slot;
    int64_t completed = 0;
    int64_t launches = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    // group requests by pattern (first-appearance order), stage inputs, enqueue copies and exec
    m2_status launch(int si, const std::vector<int64_t>& reqs) {
        Slot& sl = s->slots[si];
        sl.groups.clear();
        for (int64_t r : reqs) {
            const int pat = pattern[r];
            auto it = std::find_if(sl.groups.begin(), sl.groups.end(), [&](const Group& g) { return g.pattern == pat; });
            if (it == sl.groups.end()) {
                sl.groups.push_back(Group{});
                sl.groups.back().pattern = pat;
                it = sl.groups.end() - 1;
            }
            it->reqs.push_back(r);
        }
        size_t doff = 0, hoff = 0;
        for (Group& g : sl.groups) {
            const PlanGeo& geo = s->geo[g.pattern];
            const int64_t B = (int64_t)g.reqs.size();
            g.dx = doff;
            doff += align_up(sizeof(float) * B * geo.N);
            g.dP = doff;
            doff += align_up(sizeof(float) * B * geo.I);
            if (s->outputs & M2_OUT_J) {
                g.dJ = doff;
                doff += align_up(sizeof(float2) * B * geo.K * geo.I);
            }
            if (s->outputs & M2_OUT_E) {
                g.dE = doff;
                doff += align_up(sizeof(float) * B * geo.K * geo.I);
            }
            g.hx = hoff;
            hoff += align_up(sizeof(float) * B * geo.N);
            g.hP = hoff;
            hoff += align_up(sizeof(float) * B * geo.I);
            float* hx = reinterpret_cast<float*>(sl.host + g.hx);
            for (int64_t b = 0; b < B; ++b) std::memcpy(hx + b * geo.N, x[g.reqs[b]], sizeof(float) * geo.N);
            M2_CUDA_TRY(cudaMemcpyAsync(sl.dev + g.dx, hx, sizeof(float) * B * geo.N, cudaMemcpyHostToDevice,
                                        sl.stream));
            m2_status st = m2nufft_exec(s->plans[g.pattern], sl.dev + g.dx, B,
                                        (s->outputs & M2_OUT_J) ? sl.dev + g.dJ : nullptr,
                                        (s->outputs & M2_OUT_E) ? sl.dev + g.dE : nullptr, sl.dev + g.dP, nullptr,
                                        nullptr, sl.stream);
            if (st != M2_OK) return st;
            M2_CUDA_TRY(cudaMemcpyAsync(sl.host + g.hP, sl.dev + g.dP, sizeof(float) * B * geo.I,
                                        cudaMemcpyDeviceToHost, sl.stream));
            pattern_slot[g.pattern] = si;
        }
        M2_CUDA_TRY(cudaEventRecord(sl.done, sl.stream));
        sl.busy = true;
        ++launches;
        return M2_OK;
    }

    // all requests of the launch through the stage-batched kernels, whatever their patterns
    m2_status launch_cross(int si, const std::vector<int64_t>& reqs) {
        Slot& sl = s->slots[si];
        const int n = (int)reqs.size();
        sl.cross.clear();
        std::vector<int> plan(n);
        std::vector<const float*> xd(n);
        std::vector<float2*> Jd(n, nullptr);
        std::vector<float*> Ed(n, nullptr), Pd(n);
        // device arena: x | P | J | E | workspace | staged maps;  pinned arena: x | P | staged maps
        size_t dx = 0, hx = 0, xb = 0, pb = 0, jb = 0, eb = 0, wb = 0, mb = 0;
        for (int64_t r : reqs) {
            const PlanGeo& g = s->geo[pattern[r]];
            xb += align_up(sizeof(float) * g.N);
            pb += align_up(sizeof(float) * g.I);
            if (s->outputs & M2_OUT_J) jb += align_up(sizeof(float2) * g.K * g.I);
            if (s->outputs & M2_OUT_E) eb += align_up(sizeof(float) * g.K * g.I);
            wb += align_up(s->ws_bytes[pattern[r]]);
            mb += align_up(s->map_bytes[pattern[r]]);
        }
        const size_t dP0 = xb, dJ0 = dP0 + pb, dE0 = dJ0 + jb, dW0 = dE0 + eb, dM0 = dW0 + wb;
        const size_t hP0 = xb, hM0 = hP0 + pb;
        size_t oP = 0, oJ = 0, oE = 0;
        for (int i = 0; i < n; ++i) {
            const int64_t r = reqs[i];
            const PlanGeo& g = s->geo[pattern[r]];
            plan[i] = pattern[r];
            std::memcpy(sl.host + hx, x[r], sizeof(float) * g.N);
            xd[i] = reinterpret_cast<const float*>(sl.dev + dx);
            dx += align_up(sizeof(float) * g.N);
            hx += align_up(sizeof(float) * g.N);
            Pd[i] = reinterpret_cast<float*>(sl.dev + dP0 + oP);
            sl.cross.emplace_back(r, hP0 + oP);
            oP += align_up(sizeof(float) * g.I);
            if (s->outputs & M2_OUT_J) {
                Jd[i] = reinterpret_cast<float2*>(sl.dev + dJ0 + oJ);
                oJ += align_up(sizeof(float2) * g.K * g.I);
            }
            if (s->outputs & M2_OUT_E) {
                Ed[i] = reinterpret_cast<float*>(sl.dev + dE0 + oE);
                oE += align_up(sizeof(float) * g.K * g.I);
            }
        }
        M2_CUDA_TRY(cudaMemcpyAsync(sl.dev, sl.host, xb, cudaMemcpyHostToDevice, sl.stream));
        M2_TRY(m2::hserve_launch(s->hs, n, plan.data(), xd.data(), (s->outputs & M2_OUT_J) ? Jd.data() : nullptr,
                                 (s->outputs & M2_OUT_E) ? Ed.data() : nullptr, Pd.data(),
                                 reinterpret_cast<float2*>(sl.dev + dW0), sl.host + hM0, sl.dev + dM0, mb,
                                 sl.stream));
        M2_CUDA_TRY(cudaMemcpyAsync(sl.host + hP0, sl.dev + dP0, pb, cudaMemcpyDeviceToHost, sl.stream));
        M2_CUDA_TRY(cudaEventRecord(sl.done, sl.stream));
        sl.busy = true;
        ++launches;
        return M2_OK;
    }

    void retire(int si) {
        Slot& sl = s->slots[si];
        const double t = now();
        for (const auto& q : sl.cross) {
            const int64_t r = q.first;
            if (p_out && p_out[r])
                std::memcpy(p_out[r], sl.host + q.second, sizeof(float) * s->geo[pattern[r]].I);
            latency[r] = t - arrival[r];
            ++completed;
        }
        sl.cross.clear();
        for (const Group& g : sl.groups) {
            const PlanGeo& geo = s->geo[g.pattern];
            const float* hP = reinterpret_cast<const float*>(sl.host + g.hP);
            for (size_t b = 0; b < g.reqs.size(); ++b) {
                const int64_t r = g.reqs[b];
                if (p_out && p_out[r]) std::memcpy(p_out[r], hP + b * geo.I, sizeof(float) * geo.I);
                latency[r] = t - arrival[r];
                ++completed;
            }
            pattern_slot[g.pattern] = -1;
        }
        sl.groups.clear();
        sl.busy = false;
    }

    m2_status poll() {
        for (int si = 0; si < (int)s->slots.size(); ++si) {
            Slot& sl = s->slots[si];
            if (!sl.busy) continue;
            const cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaSuccess) {
                retire(si);
            } else if (e != cudaErrorNotReady) {
                m2::set_error("m2serve: launch failed: %s", cudaGetErrorString(e));
                return M2_ERR_CUDA;
            }
        }
        return M2_OK;
    }
};

}  // namespace

extern "C" m2_status m2serve_create(const m2nufft_plan_t* plans, int nplans, size_t mem_budget, int slots,
                                    int max_batch, unsigned outputs, m2serve_t* out) {
    m2::clear_error();
    if (!out || !plans || nplans < 1 || slots < 1 || max_batch < 1) {
        m2::set_error("m2serve_create: invalid arguments");
        return M2_ERR_ARG;
    }
    *out = nullptr;
    auto* s = new m2serve_s();
    s->outputs = (outputs & (M2_OUT_J | M2_OUT_E)) | M2_OUT_P;
    s->max_batch = max_batch;
    size_t plan_bytes = 0;
    for (int i = 0; i < nplans; ++i) {
        m2_info inf{};
        if (!plans[i] || m2nufft_get_info(plans[i], &inf) != M2_OK || inf.precision != 32) {
            delete s;
            m2::set_error("m2serve_create: plan %d is NULL or not an FP32 plan", i);
            return M2_ERR_ARG;
        }
        s->plans.push_back(plans[i]);
        s->geo.push_back(PlanGeo{inf.N, inf.I, inf.K});
        plan_bytes += inf.device_bytes;
        if (i == 0) s->device = plans[0]->device;
        if (plans[i]->device != s->device) {
            delete s;
            m2::set_error("m2serve_create: plans are on different devices");
            return M2_ERR_ARG;
        }
    }
    DevGuard guard0(s->device);
    bool all_packed = true;
    for (int i = 0; i < nplans; ++i) all_packed = all_packed && plans[i]->g.path >= 2;
    if (all_packed) {
        m2_status st = m2::hserve_create(const_cast<m2nufft_plan_s* const*>(plans), nplans, &s->hs);
        if (st != M2_OK) {
            delete s;
            return st;
        }
        for (int i = 0; i < nplans; ++i) {
            s->ws_bytes.push_back(m2::hserve_ws_bytes(s->hs, i));
            s->map_bytes.push_back(m2::hserve_map_bytes(s->hs, i));
        }
    }
    size_t max_req_dev = 0, max_req_host = 0;
    for (int i = 0; i < nplans; ++i) {
        max_req_dev = std::max(max_req_dev, s->hs ? cross_dev_bytes(s, i) : dev_bytes(s, i, 1));
        max_req_host = std::max(max_req_host, s->hs ? cross_host_bytes(s, i) : host_bytes(s, i, 1));
    }
    if (mem_budget <= plan_bytes || (mem_budget - plan_bytes) / slots < max_req_dev) {
        if (s->hs) m2::hserve_free(s->hs);
        delete s;
        m2::set_error("m2serve_create: budget %zu does not cover the plans (%zu bytes) plus one request of the "
                      "largest pattern (%zu bytes) per slot",
                      mem_budget, plan_bytes, max_req_dev);
        return M2_ERR_BUDGET;
    }
    const size_t dev_cap = std::min((mem_budget - plan_bytes) / slots, (size_t)max_batch * max_req_dev);
    const size_t host_cap = (size_t)max_batch * max_req_host;
    DevGuard guard(s->device);
    s->slots.resize(slots);
    for (Slot& sl : s->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.dev, dev_cap);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.host, host_cap);
        if (e != cudaSuccess) {
            destroy_server(s);
            m2::set_error("m2serve_create: %s", cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? M2_ERR_NOMEM : M2_ERR_CUDA;
        }
        sl.dev_cap = dev_cap;
        sl.host_cap = host_cap;
    }
    *out = s;
    return M2_OK;
}

extern "C" m2_status m2serve_run_trace(m2serve_t s, int64_t nreq, const int32_t* pattern, const double* arrival_s,
                                       const float* const* x, float* const* p_out, double* latency_s, int plain) {
    m2::clear_error();
    if (!s || nreq < 0 || (nreq > 0 && (!pattern || !arrival_s || !x || !latency_s))) {
        m2::set_error("m2serve_run_trace: invalid arguments");
        return M2_ERR_ARG;
    }
    for (int64_t r = 0; r < nreq; ++r)
        if (pattern[r] < 0 || pattern[r] >= (int32_t)s->plans.size() || !x[r]) {
            m2::set_error("m2serve_run_trace: request %lld has a bad pattern or NULL samples", (long long)r);
            return M2_ERR_ARG;
        }
    DevGuard guard(s->device);
    std::vector<int64_t> order(nreq);
    for (int64_t r = 0; r < nreq; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return arrival_s[a] < arrival_s[b]; });
    Run run{s, nreq, pattern, arrival_s, x, p_out, latency_s, Clock::now(), std::vector<int>(s->plans.size(), -1)};
    std::deque<int64_t> queue;
    int64_t next = 0;
    const int nslots = plain ? 1 : (int)s->slots.size();
    const int batch = plain ? 1 : s->max_batch;
    while (run.completed < nreq) {
        const double t = run.now();
        while (next < nreq && arrival_s[order[next]] <= t) queue.push_back(order[next++]);
        M2_TRY(run.poll());
        int free_slot = -1;
        for (int si = 0; si < nslots; ++si)
            if (!s->slots[si].busy) {
                free_slot = si;
                break;
            }
        if (free_slot >= 0 && !queue.empty()) {
            std::vector<int64_t> take;
            std::deque<int64_t> keep;
            size_t used_dev = 0, used_host = 0;
            // patterns of this launch so far, with their request counts
            std::vector<std::pair<int, int64_t>> pats;
            const bool cross = s->hs != nullptr && !plain;
            while (!queue.empty() && (int)take.size() < batch) {
                const int64_t r = queue.front();
                queue.pop_front();
                const int pat = pattern[r];
                if (cross) {  // any pattern; the slot's arena bounds the launch
                    const size_t dnew = used_dev + cross_dev_bytes(s, pat);
                    const size_t hnew = used_host + cross_host_bytes(s, pat);
                    if (dnew > s->slots[free_slot].dev_cap || hnew > s->slots[free_slot].host_cap) {
                        keep.push_back(r);
                        break;
                    }
                    used_dev = dnew;
                    used_host = hnew;
                    take.push_back(r);
                    continue;
                }
                if (run.pattern_slot[pat] >= 0) {  // pattern busy in another slot
                    keep.push_back(r);
                    continue;
                }
                auto it = std::find_if(pats.begin(), pats.end(), [&](const std::pair<int, int64_t>& q) { return q.first == pat; });
                const int64_t B = it == pats.end() ? 1 : it->second + 1;
                const size_t dnew = used_dev - (it == pats.end() ? 0 : dev_bytes(s, pat, B - 1)) + dev_bytes(s, pat, B);
                const size_t hnew = used_host - (it == pats.end() ? 0 : host_bytes(s, pat, B - 1)) + host_bytes(s, pat, B);
                if (dnew > s->slots[free_slot].dev_cap || hnew > s->slots[free_slot].host_cap) {
                    keep.push_back(r);
                    break;
                }
                used_dev = dnew;
                used_host = hnew;
                if (it == pats.end()) pats.emplace_back(pat, 1);
                else it->second += 1;
                take.push_back(r);
            }
            while (!keep.empty()) {
                queue.push_front(keep.back());
                keep.pop_back();
            }
            if (!take.empty()) {
                // a launch of one request goes through its plan's own exec (no work maps to stage
                // and upload) unless that plan's workspace is busy in another slot; both forms give
                // the same bits
                if (cross && !(take.size() == 1 && run.pattern_slot[pattern[take[0]]] < 0))
                    M2_TRY(run.launch_cross(free_slot, take));
                else M2_TRY(run.launch(free_slot, take));
                continue;
            }
        }
        bool busy = false;
        for (int si = 0; si < nslots; ++si) busy = busy || s->slots[si].busy;
        if (!busy && queue.empty() && next < nreq) {
            const double wait = arrival_s[order[next]] - run.now();
            if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
        }
    }
    s->last_launches = run.launches;
    s->last_requests = nreq;
    return M2_OK;
}

extern "C" m2_status m2serve_stats(m2serve_t s, int64_t* launches, int64_t* requests) {
    m2::clear_error();
    if (!s) {
        m2::set_error("server is NULL");
        return M2_ERR_ARG;
    }
    if (launches) *launches = s->last_launches;
    if (requests) *requests = s->last_requests;
    return M2_OK;
}

extern "C" m2_status m2serve_destroy(m2serve_t s) {
    m2::clear_error();
    destroy_server(s);
    return M2_OK;
}
