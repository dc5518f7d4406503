// Per-signal hot path of the multitaper NuFFT (Sec. 3.2, Eq. eigencoefficients
// and Eq. power_spectrum_estimator; Table 1 steps 4-5).
//
// For each chunk of signals three kernels run on the caller's stream:
//   spread  : taper-weight the samples (c_k[n] = u_k[n] x[n], kept in shared
//             memory) and gather them onto the fine grid with the
//             exponential-of-semicircle window.  Every CTA owns a tile of
//             cells and sums the contributions of the points whose window
//             covers its cells; no atomics, fixed summation order.
//   cols    : first half of a four-step FFT of length nf = n1*n2 (column
//             DFTs of length n1 over the nonzero support rows, then the
//             nf-point twiddle), written to the L2-resident workspace Z.
//   rows    : row DFTs of length n2, then the fused epilogue: deconvolve
//             and re-phase (J = X * s[i]), write J and |J|^2, and average
//             |J|^2 over the K tapers of the signal inside the CTA to form
//             P-hat without atomics.
#include <algorithm>
#include <atomic>
#include <list>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "common.cuh"

namespace m2 {

m2_status check_stage_status(m2nufft_plan_s* p) {
    int* h = p->stage_status;
    if (h && ((volatile int*)h)[0] != 0) {
        const int where = ((volatile int*)h)[2];
        h[0] = h[1] = h[2] = 0;
        set_error("an earlier launch of a packed stage kernel gave up waiting for a bulk copy (spread tile %d; "
                  "M2_ERR_TIMEOUT)", where);
        return M2_ERR_TIMEOUT;
    }
    return M2_OK;
}

namespace {

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) {
    C r;
    r.x = a.x + b.x;
    r.y = a.y + b.y;
    return r;
}
template <typename C> __device__ __forceinline__ C csub(C a, C b) {
    C r;
    r.x = a.x - b.x;
    r.y = a.y - b.y;
    return r;
}
// a * (-i)
template <typename C> __device__ __forceinline__ C cmul_mi(C a) {
    C r;
    r.x = a.y;
    r.y = -a.x;
    return r;
}

__device__ __forceinline__ float es_kernel(float z, float two_over_w, float beta) {
    float a = z * two_over_w;
    float s = fmaxf(0.0f, 1.0f - a * a);
    return expf(beta * (sqrtf(s) - 1.0f));
}
__device__ __forceinline__ double es_kernel(double z, double two_over_w, double beta) {
    double a = z * two_over_w;
    double s = fmax(0.0, 1.0 - a * a);
    return exp(beta * (sqrt(s) - 1.0));
}

__device__ __forceinline__ int bitrev(int v, int bits) {
    return (int)(__brev((unsigned)v) >> (32 - bits));
}

// In-place radix-2/4 decimation-in-time FFTs of `nrows` rows of length M
// (row stride `rs` elements) in shared memory.  Input must be in
// bit-reversed order; output is in natural order.  `tw[q]` = exp(-i 2 pi q/M)
// for q < M/2.  Caller synchronises before (data ready) and after.
template <typename C>
__device__ void fft_rows_dit(C* buf, int nrows, int M, int logM, int rs, const C* tw) {
    const int nt = blockDim.x;
    int s = 0;
    if (logM & 1) {
        const int half = M >> 1;
        for (int idx = threadIdx.x; idx < nrows * half; idx += nt) {
            int r = idx / half, j = idx - r * half;
            C* b = buf + r * rs + 2 * j;
            C a = b[0], c = b[1];
            b[0] = cadd(a, c);
            b[1] = csub(a, c);
        }
        s = 1;
        __syncthreads();
    }
    for (; s < logM; s += 2) {
        const int h = 1 << s;
        const int quarter = M >> 2;
        const int sh1 = logM - s - 1, sh2 = logM - s - 2;
        for (int idx = threadIdx.x; idx < nrows * quarter; idx += nt) {
            int r = idx / quarter, q = idx - r * quarter;
            int blk = q >> s, rr = q & (h - 1);
            C* b = buf + r * rs + blk * 4 * h + rr;
            C x0 = b[0], x1 = b[h], x2 = b[2 * h], x3 = b[3 * h];
            C w1 = tw[rr << sh1];
            C t1 = cmul(x1, w1), t3 = cmul(x3, w1);
            C a0 = cadd(x0, t1), a1 = csub(x0, t1), a2 = cadd(x2, t3), a3 = csub(x2, t3);
            C w2 = tw[rr << sh2];
            C u2 = cmul(a2, w2), u3 = cmul_mi(cmul(a3, w2));
            b[0] = cadd(a0, u2);
            b[2 * h] = csub(a0, u2);
            b[h] = cadd(a1, u3);
            b[3 * h] = csub(a1, u3);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// spread: g[b][k][c] = sum_n u_k[n] x_b[n] phi(c - u_n)
// ---------------------------------------------------------------------------
template <typename R, bool CPLX, int KM>
__global__ void __launch_bounds__(kSpreadTile)
spread_kernel(const R* __restrict__ x, int64_t N, const int32_t* __restrict__ pt_src,
              const int32_t* __restrict__ pt_cell, const R* __restrict__ pt_off,
              const void* __restrict__ taper_v, int64_t P, const int32_t* __restrict__ tile_pb,
              const int32_t* __restrict__ tile_pe, int K, int w, R two_over_w, R beta, int64_t Lg,
              typename CT<R>::C* __restrict__ g) {
    using C = typename CT<R>::C;
    using V = typename std::conditional<CPLX, C, R>::type;
    extern __shared__ unsigned char smem_raw[];
    int32_t* s_cell = reinterpret_cast<int32_t*>(smem_raw);
    R* s_off = reinterpret_cast<R*>(smem_raw + sizeof(R) * kSpreadChunk);  // aligned: chunk*8 bytes
    V* s_val = reinterpret_cast<V*>(smem_raw + 2 * sizeof(R) * kSpreadChunk);

    const V* taper = reinterpret_cast<const V*>(taper_v);
    const int tile = blockIdx.x;
    const int b = blockIdx.y;
    const int64_t c = (int64_t)tile * kSpreadTile + threadIdx.x;
    const int pb = tile_pb[tile], pe = tile_pe[tile];
    const R* xb = x + (int64_t)b * N;

    C acc[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) acc[k].x = acc[k].y = R(0);

    for (int q0 = pb; q0 < pe; q0 += kSpreadChunk) {
        const int n = min(kSpreadChunk, pe - q0);
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const int p = q0 + j;
            s_cell[j] = pt_cell[p];
            s_off[j] = pt_off[p];
            const R xv = xb[pt_src[p]];
            for (int k = 0; k < K; ++k) {
                V tv = taper[(int64_t)k * P + p];
                if constexpr (CPLX) {
                    tv.x *= xv;
                    tv.y *= xv;
                } else {
                    tv *= xv;
                }
                s_val[k * kSpreadChunk + j] = tv;
            }
        }
        __syncthreads();
        if (c < Lg) {
            const int ci = (int)c;
            // first staged point whose window reaches cell c
            int lo = 0, hi = n;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (s_cell[mid] + w <= ci) lo = mid + 1; else hi = mid;
            }
            for (int j = lo; j < n && s_cell[j] <= ci; ++j) {
                const R z = s_off[j] + (R)(ci - s_cell[j]);
                const R phi = es_kernel(z, two_over_w, beta);
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    if (k < K) {
                        V v = s_val[k * kSpreadChunk + j];
                        if constexpr (CPLX) {
                            acc[k].x += v.x * phi;
                            acc[k].y += v.y * phi;
                        } else {
                            acc[k].x += v * phi;
                        }
                    }
                }
            }
        }
    }
    if (c < Lg) {
#pragma unroll
        for (int k = 0; k < KM; ++k)
            if (k < K) g[((int64_t)b * K + k) * Lg + c] = acc[k];
    }
}

// ---------------------------------------------------------------------------
// column pass: Z[b][k][k1][l2] = W_nf^{l2 k1} sum_{l1 < rows} g[b][k][n2 l1 + l2] W_n1^{l1 k1}
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
cols_kernel(const typename CT<R>::C* __restrict__ g, int64_t Lg, int rows, int n1, int log_n1,
            int n2, int cw, int K, const typename CT<R>::C* __restrict__ tw1,
            const typename CT<R>::C* __restrict__ twa, const typename CT<R>::C* __restrict__ twb,
            int twb_bits, typename CT<R>::C* __restrict__ Z) {
    using C = typename CT<R>::C;
    extern __shared__ unsigned char smem_raw[];
    C* s_tw = reinterpret_cast<C*>(smem_raw);
    C* buf = s_tw + (n1 >> 1);
    const int rs = n1 + 1;

    const int c0 = blockIdx.x * cw;
    const int k = blockIdx.y;
    const int b = blockIdx.z;
    const C* gk = g + ((int64_t)b * K + k) * Lg;
    C* Zk = Z + ((int64_t)b * K + k) * (int64_t)n1 * n2;

    for (int q = threadIdx.x; q < (n1 >> 1); q += blockDim.x) s_tw[q] = tw1[q];
    const int total = n1 * cw;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int l1 = idx / cw, c = idx - l1 * cw;
        C v;
        if (l1 < rows) v = gk[(int64_t)l1 * n2 + c0 + c];
        else v.x = v.y = R(0);
        buf[c * rs + bitrev(l1, log_n1)] = v;
    }
    __syncthreads();
    fft_rows_dit(buf, cw, n1, log_n1, rs, s_tw);
    const int lmask = (1 << twb_bits) - 1;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int k1 = idx / cw, c = idx - k1 * cw;
        const int l2 = c0 + c;
        const int64_t q = (int64_t)l2 * k1;  // < nf
        const C tw = cmul(twa[q >> twb_bits], twb[q & lmask]);
        Zk[(int64_t)k1 * n2 + l2] = cmul(buf[c * rs + k1], tw);
    }
}

// ---------------------------------------------------------------------------
// row pass + epilogue
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
rows_kernel(const typename CT<R>::C* __restrict__ Z, int n1, int n2, int log_n2, int rw, int K,
            int64_t I, int64_t i_c, int64_t nf, const typename CT<R>::C* __restrict__ tw2,
            const typename CT<R>::C* __restrict__ deconv, typename CT<R>::C* __restrict__ J,
            R* __restrict__ E, R* __restrict__ Pout) {
    using C = typename CT<R>::C;
    extern __shared__ unsigned char smem_raw[];
    C* s_tw = reinterpret_cast<C*>(smem_raw);
    C* buf = s_tw + (n2 >> 1);
    const int rs = n2 + 1;
    R* pacc = reinterpret_cast<R*>(buf + rw * rs);

    const int r0 = blockIdx.x * rw;
    const int b = blockIdx.y;
    const int total = rw * n2;
    const int64_t half = nf >> 1;

    for (int q = threadIdx.x; q < (n2 >> 1); q += blockDim.x) s_tw[q] = tw2[q];
    for (int e = threadIdx.x; e < total; e += blockDim.x) pacc[e] = R(0);

    for (int k = 0; k < K; ++k) {
        const C* Zk = Z + ((int64_t)b * K + k) * (int64_t)n1 * n2;
        __syncthreads();
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int r = idx / n2, l2 = idx - r * n2;
            buf[r * rs + bitrev(l2, log_n2)] = Zk[(int64_t)(r0 + r) * n2 + l2];
        }
        __syncthreads();
        fft_rows_dit(buf, rw, n2, log_n2, rs, s_tw);
        C* Jk = J ? J + ((int64_t)b * K + k) * I : nullptr;
        R* Ek = E ? E + ((int64_t)b * K + k) * I : nullptr;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int r = e % rw, k2 = e / rw;
            const int64_t kk = (int64_t)(r0 + r) + (int64_t)n1 * k2;
            const int64_t m = kk < half ? kk : kk - nf;
            const int64_t i = m + i_c;
            if (i >= 0 && i < I) {
                const C jv = cmul(buf[r * rs + k2], deconv[i]);
                const R p = jv.x * jv.x + jv.y * jv.y;
                if (Jk) Jk[i] = jv;
                if (Ek) Ek[i] = p;
                pacc[e] += p;
            }
        }
    }
    if (Pout) {
        __syncthreads();
        const R invK = R(1) / (R)K;
        R* Pb = Pout + (int64_t)b * I;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int r = e % rw, k2 = e / rw;
            const int64_t kk = (int64_t)(r0 + r) + (int64_t)n1 * k2;
            const int64_t m = kk < half ? kk : kk - nf;
            const int64_t i = m + i_c;
            if (i >= 0 && i < I) Pb[i] = pacc[e] * invK;
        }
    }
}

template <typename R>
size_t spread_smem(int K, bool cplx) {
    return 2 * sizeof(R) * kSpreadChunk +
           (size_t)K * kSpreadChunk * (cplx ? 2 * sizeof(R) : sizeof(R));
}
template <typename R>
size_t cols_smem(const Geometry& g) {
    using C = typename CT<R>::C;
    return sizeof(C) * ((size_t)(g.n1 >> 1) + (size_t)g.cw * (g.n1 + 1));
}
template <typename R>
size_t rows_smem(const Geometry& g) {
    using C = typename CT<R>::C;
    return sizeof(C) * ((size_t)(g.n2 >> 1) + (size_t)g.rw * (g.n2 + 1)) +
           sizeof(R) * (size_t)g.rw * g.n2;
}

template <typename R, bool CPLX, int KM>
m2_status launch_spread(const m2nufft_plan_s* p, const R* x, int nb, cudaStream_t st) {
    using C = typename CT<R>::C;
    const Geometry& g = p->g;
    const size_t smem = spread_smem<R>(g.K, CPLX);
    auto kern = spread_kernel<R, CPLX, KM>;
    dim3 grid((unsigned)g.ntiles, (unsigned)nb);
    kern<<<grid, kSpreadTile, smem, st>>>(
        x, g.N, p->d_pt_src, p->d_pt_cell, reinterpret_cast<const R*>(p->d_pt_off), p->d_taper, g.P,
        p->d_tile_pb, p->d_tile_pe, g.K, g.width, (R)(2.0 / g.width), (R)g.beta, g.Lg,
        reinterpret_cast<C*>(p->d_g));
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

template <typename R, bool CPLX>
m2_status launch_spread_k(const m2nufft_plan_s* p, const R* x, int nb, cudaStream_t st) {
    const int K = p->g.K;
    if (K <= 4) return launch_spread<R, CPLX, 4>(p, x, nb, st);
    if (K <= 8) return launch_spread<R, CPLX, 8>(p, x, nb, st);
    return launch_spread<R, CPLX, 16>(p, x, nb, st);
}

template <typename R>
m2_status exec_chunk(m2nufft_plan_s* p, const R* x, int nb, typename CT<R>::C* J, R* E, R* P,
                     cudaStream_t st) {
    using C = typename CT<R>::C;
    const Geometry& g = p->g;
    mark(p, 0, 0, st);
    if (g.real_taper) M2_TRY((launch_spread_k<R, false>(p, x, nb, st)));
    else M2_TRY((launch_spread_k<R, true>(p, x, nb, st)));
    mark(p, 0, 1, st);

    {
        const size_t smem = cols_smem<R>(g);
        auto kern = cols_kernel<R>;
        dim3 grid((unsigned)(g.n2 / g.cw), (unsigned)g.K, (unsigned)nb);
        mark(p, 1, 0, st);
        kern<<<grid, 256, smem, st>>>(reinterpret_cast<const C*>(p->d_g), g.Lg, (int)g.rows, (int)g.n1,
                                      g.log_n1, (int)g.n2, g.cw, g.K,
                                      reinterpret_cast<const C*>(p->d_tw1),
                                      reinterpret_cast<const C*>(p->d_twa),
                                      reinterpret_cast<const C*>(p->d_twb), g.twb_bits,
                                      reinterpret_cast<C*>(p->d_Z));
        M2_CUDA_TRY(cudaGetLastError());
        mark(p, 1, 1, st);
    }
    {
        const size_t smem = rows_smem<R>(g);
        auto kern = rows_kernel<R>;
        dim3 grid((unsigned)(g.n1 / g.rw), (unsigned)nb);
        mark(p, 2, 0, st);
        kern<<<grid, 256, smem, st>>>(reinterpret_cast<const C*>(p->d_Z), (int)g.n1, (int)g.n2, g.log_n2,
                                      g.rw, g.K, g.I, g.i_c, g.nf,
                                      reinterpret_cast<const C*>(p->d_tw2),
                                      reinterpret_cast<const C*>(p->d_deconv), J, E, P);
        M2_CUDA_TRY(cudaGetLastError());
        mark(p, 2, 1, st);
    }
    return M2_OK;
}

// Workspaces of lanes 1 .. kLanes - 1 and the internal streams of a packed plan, created on first
// use (an exec of more than one chunk; never during stream capture, where B = 1).
m2_status ensure_lanes(m2nufft_plan_s* p) {
    if (p->lane_st[0]) return M2_OK;
    const Geometry& g = p->g;
    const size_t ng = (size_t)g.chunk * g.kp * g.Lg, nz = (size_t)g.chunk * g.kp * g.nf;
    p->lane_g[0] = p->d_g;
    p->lane_Z[0] = p->d_Z;
    for (int L = 1; L < kLanes; ++L) {
        void *a = nullptr, *b = nullptr;
        M2_CUDA_TRY(cudaMalloc(&a, sizeof(float2) * ng));
        p->allocations.push_back(a);
        M2_CUDA_TRY(cudaMalloc(&b, sizeof(float2) * nz));
        p->allocations.push_back(b);
        p->device_bytes += sizeof(float2) * (ng + nz);
        p->lane_g[L] = a;
        p->lane_Z[L] = b;
    }
    M2_CUDA_TRY(cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming));
    for (int L = 0; L < kLanes; ++L) {
        M2_CUDA_TRY(cudaStreamCreateWithFlags(&p->lane_st[L], cudaStreamNonBlocking));
        M2_CUDA_TRY(cudaEventCreateWithFlags(&p->lane_ev[L], cudaEventDisableTiming));
    }
    return M2_OK;
}

// Thomson's F-statistic (Sec. 3, Eq. f_stat) from the eigencoefficients of nb signals, generic
// path: thread = band i of signal b;  C = sum_k J_k W_k / sum_k W_k^2,
// F = |C|^2 (K - 1) sum_k W_k^2 / sum_k |J_k - C W_k|^2.
template <typename R>
__global__ void __launch_bounds__(128) ftest_kernel(const typename CT<R>::C* __restrict__ J, int K, int64_t I,
                                                    const R* __restrict__ wsum, R wq, R* __restrict__ F) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= I) return;
    const auto* Jb = J + (int64_t)b * K * I + i;
    R sx = 0, sy = 0;
    for (int k = 0; k < K; ++k) {
        const auto v = Jb[(int64_t)k * I];
        sx += v.x * wsum[k];
        sy += v.y * wsum[k];
    }
    const R cx = sx / wq, cy = sy / wq;
    R res = 0;
    for (int k = 0; k < K; ++k) {
        const auto v = Jb[(int64_t)k * I];
        const R rx = v.x - cx * wsum[k], ry = v.y - cy * wsum[k];
        res += rx * rx + ry * ry;
    }
    F[(int64_t)b * I + i] = (cx * cx + cy * cy) * (R)(K - 1) * wq / res;
}

// The generic path forms F from J: a chunk-sized J buffer for calls that want F but no J,
// allocated on first use (before a batch capture by exec_batch).
m2_status prepare_jscratch(m2nufft_plan_s* p) {
    if (p->d_Jscratch) return M2_OK;
    const Geometry& g = p->g;
    const size_t bytes = (p->precision == 32 ? sizeof(float2) : sizeof(double2)) * (size_t)g.chunk * g.K * g.I;
    M2_CUDA_TRY(cudaMalloc(&p->d_Jscratch, bytes));
    p->allocations.push_back(p->d_Jscratch);
    p->device_bytes += bytes;
    return M2_OK;
}

template <typename R>
m2_status exec_typed(m2nufft_plan_s* p, const void* xv, int64_t B, void* Jv, void* Ev, void* Pv, void* Fv,
                     cudaStream_t st) {
    using C = typename CT<R>::C;
    const Geometry& g = p->g;
    const R* x = reinterpret_cast<const R*>(xv);
    C* J = reinterpret_cast<C*>(Jv);
    R* E = reinterpret_cast<R*>(Ev);
    R* P = reinterpret_cast<R*>(Pv);
    R* F = reinterpret_cast<R*>(Fv);
    if constexpr (std::is_same<R, float>::value) {
        // all B signals in one launch; the F-statistic runs the four-kernel form (same stages)
        if (g.path == 3 && !F) return exec_pipe(p, x, B, J, E, P, st);
    }
    if (F && g.path == 1 && !J) M2_TRY(prepare_jscratch(p));
    const float2* gall = nullptr;
    if constexpr (std::is_same<R, float>::value) {
        // multi-chunk execs of the packed path: the spread grids of all signals in one launch (the
        // spread is a fixed-latency chain of dependent loads, cheaper once than once per chunk),
        // while they fit in 256 MiB
        if (g.path >= 2 && B > g.chunk) {
            const size_t gsig = sizeof(float2) * (size_t)g.kp * (size_t)g.Lg;
            if ((size_t)B * gsig <= (size_t(256) << 20)) {
                if (p->gall_signals < B) {
                    if (p->d_gall) {
                        // growing (rare): the last exec that read the old buffer (every reader is
                        // joined back to its caller's stream before gall_ev is recorded there) must
                        // be done before it is freed; other plans and streams are not waited for
                        M2_CUDA_TRY(cudaEventSynchronize(p->gall_ev));
                        cudaFree(p->d_gall);
                        p->device_bytes -= gsig * (size_t)p->gall_signals;
                        p->d_gall = nullptr;
                        p->gall_signals = 0;
                    }
                    if (!p->gall_ev) M2_CUDA_TRY(cudaEventCreateWithFlags(&p->gall_ev, cudaEventDisableTiming));
                    M2_CUDA_TRY(cudaMalloc(&p->d_gall, gsig * (size_t)B));
                    p->gall_signals = B;
                    p->device_bytes += gsig * (size_t)B;
                }
                mark(p, 0, 0, st);
                M2_TRY(spread_fast(p, x, (int)B, reinterpret_cast<float2*>(p->d_gall), st));
                mark(p, 0, 1, st);
                gall = reinterpret_cast<const float2*>(p->d_gall);
            }
        }
        if (g.path >= 2 && B > g.chunk && !p->timing) {
            // kLanes lanes: chunk c on lane c % kLanes with that lane's workspace, forked from and
            // joined back to the caller's stream
            M2_TRY(ensure_lanes(p));
            M2_CUDA_TRY(cudaEventRecord(p->fork_ev, st));
            for (int L = 0; L < kLanes; ++L) M2_CUDA_TRY(cudaStreamWaitEvent(p->lane_st[L], p->fork_ev, 0));
            int c = 0;
            for (int64_t b0 = 0; b0 < B; b0 += g.chunk, ++c) {
                const int nb = (int)std::min<int64_t>(g.chunk, B - b0);
                M2_TRY(exec_fast_chunk(p, x + b0 * g.N, nb, J ? J + b0 * g.K * g.I : nullptr,
                                       E ? E + b0 * g.K * g.I : nullptr, P ? P + b0 * g.I : nullptr,
                                       F ? F + b0 * g.I : nullptr, p->lane_st[c % kLanes], c % kLanes,
                                       gall ? gall + b0 * g.kp * g.Lg : nullptr));
            }
            for (int L = 0; L < kLanes; ++L) {
                M2_CUDA_TRY(cudaEventRecord(p->lane_ev[L], p->lane_st[L]));
                M2_CUDA_TRY(cudaStreamWaitEvent(st, p->lane_ev[L], 0));
            }
            if (gall) M2_CUDA_TRY(cudaEventRecord(p->gall_ev, st));
            return M2_OK;
        }
    }
    for (int64_t b0 = 0; b0 < B; b0 += g.chunk) {
        const int nb = (int)std::min<int64_t>(g.chunk, B - b0);
        C* Jc = J ? J + b0 * g.K * g.I : nullptr;
        R* Ec = E ? E + b0 * g.K * g.I : nullptr;
        R* Pc = P ? P + b0 * g.I : nullptr;
        R* Fc = F ? F + b0 * g.I : nullptr;
        if constexpr (std::is_same<R, float>::value) {
            if (g.path >= 2) {
                M2_TRY(exec_fast_chunk(p, x + b0 * g.N, nb, Jc, Ec, Pc, Fc, st, 0,
                                       gall ? gall + b0 * g.kp * g.Lg : nullptr));
                continue;
            }
        }
        if (Fc && !Jc) Jc = reinterpret_cast<C*>(p->d_Jscratch);
        M2_TRY(exec_chunk<R>(p, x + b0 * g.N, nb, Jc, Ec, Pc, st));
        if (Fc) {
            dim3 grid((unsigned)((g.I + 127) / 128), (unsigned)nb);
            ftest_kernel<R><<<grid, 128, 0, st>>>(Jc, g.K, g.I, reinterpret_cast<const R*>(p->d_wsum), (R)p->wq, Fc);
            M2_CUDA_TRY(cudaGetLastError());
        }
    }
    if (gall) M2_CUDA_TRY(cudaEventRecord(p->gall_ev, st));
    return M2_OK;
}

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

m2_status exec_one(m2nufft_plan_s* p, const void* x, int64_t B, void* J, void* E, void* P, void* F,
                   double* Lhat, double* Ehat, cudaStream_t st) {
    if (B < 0) {
        set_error("m2nufft_exec: B must be >= 0");
        return M2_ERR_ARG;
    }
    if ((Lhat || Ehat) && !p->have_leakage) {
        set_error("m2nufft_exec: L-hat/E-hat are not available for this plan "
                  "(no eigenvalues were supplied, or the sampling pattern needs the general leakage path)");
        return M2_ERR_ARG;
    }
    if (B > 0 && !x) {
        set_error("m2nufft_exec: x is NULL");
        return M2_ERR_ARG;
    }
    if (F && p->g.K < 2) {
        set_error("m2nufft_exec_ftest: the F-statistic needs K >= 2 tapers (F(2, 2K - 2))");
        return M2_ERR_ARG;
    }
    if (F && p->complex_taper) {
        set_error("m2nufft_exec_ftest: the F-statistic is formed for full-band plans (real tapers, f_c0 = 0)");
        return M2_ERR_ARG;
    }
    M2_TRY(check_stage_status(p));
    if (B > 0) {
        if (p->precision == 32) M2_TRY(exec_typed<float>(p, x, B, J, E, P, F, st));
        else M2_TRY(exec_typed<double>(p, x, B, J, E, P, F, st));
    }
    const Geometry& g = p->g;
    if (Lhat)
        M2_CUDA_TRY(cudaMemcpyAsync(Lhat, p->d_Lhat, sizeof(double) * g.K * g.I, cudaMemcpyDefault, st));
    if (Ehat)
        M2_CUDA_TRY(cudaMemcpyAsync(Ehat, p->d_Ehat, sizeof(double) * g.I, cudaMemcpyDefault, st));
    return M2_OK;
}

}  // namespace

// Raise the dynamic shared-memory limit of every generic exec kernel to the device's opt-in
// maximum, once per device (so no launch needs an attribute call).
m2_status init_exec_kernels(int smem_optin) {
    const void* funcs[] = {
        (const void*)spread_kernel<float, false, 4>,  (const void*)spread_kernel<float, false, 8>,
        (const void*)spread_kernel<float, false, 16>, (const void*)spread_kernel<float, true, 4>,
        (const void*)spread_kernel<float, true, 8>,   (const void*)spread_kernel<float, true, 16>,
        (const void*)spread_kernel<double, false, 4>, (const void*)spread_kernel<double, false, 8>,
        (const void*)spread_kernel<double, false, 16>, (const void*)spread_kernel<double, true, 4>,
        (const void*)spread_kernel<double, true, 8>,  (const void*)spread_kernel<double, true, 16>,
        (const void*)cols_kernel<float>,              (const void*)cols_kernel<double>,
        (const void*)rows_kernel<float>,              (const void*)rows_kernel<double>,
    };
    for (const void* f : funcs)
        M2_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin));
    return M2_OK;
}

cudaEvent_t take_event(m2nufft_plan_s* p) {
    cudaEvent_t e = nullptr;
    if (!p->ev_pool.empty()) {
        e = p->ev_pool.back();
        p->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

void mark(m2nufft_plan_s* p, int kernel, int which, cudaStream_t st) {
    if (!p->timing) return;
    cudaEvent_t e = take_event(p);
    if (!e) return;
    cudaEventRecord(e, st);
    p->ev_rec[kernel][which].push_back(e);
}

}  // namespace m2

extern "C" m2_status m2nufft_exec(m2nufft_plan_t p, const void* x, int64_t B, void* J, void* E, void* P,
                                  double* Lhat, double* Ehat, void* stream) {
    m2::clear_error();
    if (!p) {
        m2::set_error("m2nufft_exec: plan is NULL");
        return M2_ERR_ARG;
    }
    m2::DeviceGuard guard(p->device);
    return m2::exec_one(p, x, B, J, E, P, nullptr, Lhat, Ehat, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" m2_status m2nufft_exec_ftest(m2nufft_plan_t p, const void* x, int64_t B, void* J, void* E, void* P,
                                        void* F, void* stream) {
    m2::clear_error();
    if (!p || !F) {
        m2::set_error("m2nufft_exec_ftest: plan or F is NULL");
        return M2_ERR_ARG;
    }
    m2::DeviceGuard guard(p->device);
    return m2::exec_one(p, x, B, J, E, P, F, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

namespace m2 {
namespace {

// Uneven batches run as one cached CUDA graph: the per-signal work is captured with signals of
// different plans on different internal streams (signals of one plan share a stream, since they
// share that plan's workspace), joined back, instantiated once per distinct (plans, buffers)
// key, and replayed with one cudaGraphLaunch on the caller's stream.
constexpr int kBatchStreams = 8;
constexpr size_t kMaxGraphs = 16;

struct BatchResources {
    bool ready = false;
    cudaStream_t origin = nullptr;
    cudaStream_t ws[kBatchStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kBatchStreams] = {};
};

struct GraphEntry {
    int device;
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec;
    PipeLaunch* pipe;  // persistent-kernel batch (owned), or NULL
    HBatch* hb;        // stage-batched batch (owned), or NULL
};

void drop_entry(GraphEntry& e) {
    cudaGraphExecDestroy(e.exec);
    if (e.pipe) pipe_free(e.pipe);
    if (e.hb) hbatch_free(e.hb);
}

// How all-packed batches run: 0 = stage-batched launches, 1 = one persistent-kernel launch,
// 2 = whichever form and stage-batched CTA shapes measured fastest for the batch (tuned on the
// first call for the batch's signature, then cached with its graph).
std::atomic<int> g_batch_mode{0};

// The candidates and their measured times of the most recently tuned batch (guarded by g_batch_mu).
struct BatchTuneRow {
    int mode;
    HBConfig cfg;
    double ms;
};
std::vector<BatchTuneRow> g_batch_tuning;

std::mutex g_batch_mu;
BatchResources g_batch_res[64];
std::list<GraphEntry> g_graphs;  // most recently used first

m2_status batch_resources(int dev, BatchResources** out) {
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return M2_ERR_ARG;
    }
    BatchResources& r = g_batch_res[dev];
    if (!r.ready) {
        M2_CUDA_TRY(cudaStreamCreateWithFlags(&r.origin, cudaStreamNonBlocking));
        M2_CUDA_TRY(cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming));
        for (int w = 0; w < kBatchStreams; ++w) {
            M2_CUDA_TRY(cudaStreamCreateWithFlags(&r.ws[w], cudaStreamNonBlocking));
            M2_CUDA_TRY(cudaEventCreateWithFlags(&r.join[w], cudaEventDisableTiming));
        }
        r.ready = true;
    }
    *out = &r;
    return M2_OK;
}

m2_status capture_batch(const m2nufft_plan_t* plans, const void* const* xs, int64_t nsig, void* const* Js,
                        void* const* Es, void* const* Ps, void* const* Fs, BatchResources& r, cudaGraphExec_t* out) {
    // stream of each distinct plan, round robin in order of first appearance
    std::unordered_map<const m2nufft_plan_s*, int> lane;
    for (int64_t s = 0; s < nsig; ++s)
        if (!lane.count(plans[s])) lane.emplace(plans[s], (int)(lane.size() % kBatchStreams));
    // launch configurations of pipelined plans, and the J buffers of generic plans asked for F
    // without J, are created before the capture (they allocate)
    for (const auto& kv : lane)
        if (kv.first->g.path == 3) M2_TRY(pipe_prepare(const_cast<m2nufft_plan_s*>(kv.first), 1));
    for (int64_t s = 0; s < nsig; ++s)
        if (Fs && Fs[s] && plans[s]->g.path == 1 && !(Js && Js[s])) M2_TRY(prepare_jscratch(plans[s]));
    M2_CUDA_TRY(cudaStreamBeginCapture(r.origin, cudaStreamCaptureModeThreadLocal));
    m2_status st = M2_OK;
    cudaError_t e = cudaEventRecord(r.fork, r.origin);
    for (int w = 0; w < kBatchStreams && e == cudaSuccess; ++w) e = cudaStreamWaitEvent(r.ws[w], r.fork, 0);
    if (e != cudaSuccess) {
        set_error("batch capture fork failed: %s", cudaGetErrorString(e));
        st = M2_ERR_CUDA;
    }
    for (int64_t s = 0; s < nsig && st == M2_OK; ++s) {
        m2nufft_plan_s* p = plans[s];
        const int saved = p->timing;
        p->timing = 0;
        st = exec_one(p, xs[s], 1, Js ? Js[s] : nullptr, Es ? Es[s] : nullptr, Ps ? Ps[s] : nullptr,
                      Fs ? Fs[s] : nullptr, nullptr, nullptr, r.ws[lane[p]]);
        p->timing = saved;
    }
    // the worker streams are joined back even after a failure, so that ending the capture leaves
    // none of them capturing
    for (int w = 0; w < kBatchStreams; ++w) {
        e = cudaEventRecord(r.join[w], r.ws[w]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(r.origin, r.join[w], 0);
        if (e != cudaSuccess && st == M2_OK) {
            set_error("batch capture join failed: %s", cudaGetErrorString(e));
            st = M2_ERR_CUDA;
        }
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(r.origin, &graph);
    if (st == M2_OK && e != cudaSuccess) {
        set_error("cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
        st = M2_ERR_CUDA;
    }
    if (st == M2_OK) {
        e = cudaGraphInstantiate(out, graph, 0);
        if (e != cudaSuccess) {
            set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
            st = M2_ERR_CUDA;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != M2_OK) (void)cudaGetLastError();  // reported: not again by a later launch check
    return st;
}

// All-packed batch: the persistent-kernel launch (counter reset + kernel), or the stage-batched
// launches, captured as a graph.
m2_status capture_packed_batch(PipeLaunch* L, HBatch* H, BatchResources& r, cudaGraphExec_t* out) {
    M2_CUDA_TRY(cudaStreamBeginCapture(r.origin, cudaStreamCaptureModeThreadLocal));
    m2_status st = L ? pipe_batch_run(L, r.origin) : hbatch_run(H, r.origin);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(r.origin, &graph);
    if (st == M2_OK && e != cudaSuccess) {
        set_error("cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
        st = M2_ERR_CUDA;
    }
    if (st == M2_OK) {
        e = cudaGraphInstantiate(out, graph, 0);
        if (e != cudaSuccess) {
            set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
            st = M2_ERR_CUDA;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != M2_OK) (void)cudaGetLastError();  // reported: not again by a later launch check
    return st;
}

// Tuning of an all-packed batch: every stage-batched CTA shape (spread tiles per CTA 1 / 2 / 4,
// rows per CTA 8 / 4, epilogue tiles 32 x 16 / 16 x 16) and the persistent kernel are built,
// captured and timed on `st` (one warm-up launch, then the mean of three, CUDA events); the
// fastest is kept (its resources returned), the others freed.  Every candidate writes the same
// bits.  With F-statistic outputs the persistent kernel (which forms none) is not a candidate.
// Synchronous; not allowed while `st` is capturing.
m2_status tune_packed_batch(m2nufft_plan_s* const* plans, const void* const* xs, int64_t nsig, void* const* Js,
                            void* const* Es, void* const* Ps, void* const* Fs, BatchResources& r, cudaStream_t st,
                            cudaGraphExec_t* out, PipeLaunch** out_pipe, HBatch** out_hb) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    M2_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        set_error("m2nufft_exec_batch: batch mode 2 tunes on the first call for a batch, which cannot be captured");
        return M2_ERR_ARG;
    }
    std::vector<std::pair<int, HBConfig>> cands;
    for (int nt : {1, 2, 4})
        for (int rw : {8, 4})
            for (int t1 : {32, 16}) cands.push_back({0, HBConfig{nt, rw, t1}});
    if (!Fs) cands.push_back({1, HBConfig{}});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    M2_CUDA_TRY(cudaEventCreate(&e0));
    M2_CUDA_TRY(cudaEventCreate(&e1));
    std::vector<BatchTuneRow> rows;
    double best_ms = 1e300;
    cudaGraphExec_t best = nullptr;
    PipeLaunch* best_pipe = nullptr;
    HBatch* best_hb = nullptr;
    m2_status status = M2_OK;
    for (const auto& c : cands) {
        PipeLaunch* pipe = nullptr;
        HBatch* hb = nullptr;
        cudaGraphExec_t ex = nullptr;
        status = c.first == 1 ? pipe_batch_create(plans, xs, nsig, Js, Es, Ps, &pipe)
                              : hbatch_create(plans, xs, nsig, Js, Es, Ps, Fs, c.second, &hb);
        if (status == M2_OK) status = capture_packed_batch(pipe, hb, r, &ex);
        float ms = 0.f;
        cudaError_t e = cudaSuccess;
        if (status == M2_OK) {
            e = cudaGraphLaunch(ex, st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaGraphLaunch(ex, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                set_error("m2nufft_exec_batch tuning: %s", cudaGetErrorString(e));
                status = M2_ERR_CUDA;
            }
            if (status == M2_OK && pipe) status = pipe_check(pipe);
        }
        const double t = ms / 3.0;
        if (status == M2_OK) rows.push_back(BatchTuneRow{c.first, c.second, t});
        if (status == M2_OK && t < best_ms) {
            if (best) cudaGraphExecDestroy(best);
            if (best_pipe) pipe_free(best_pipe);
            if (best_hb) hbatch_free(best_hb);
            best_ms = t;
            best = ex;
            best_pipe = pipe;
            best_hb = hb;
        } else {
            if (ex) cudaGraphExecDestroy(ex);
            if (pipe) pipe_free(pipe);
            if (hb) hbatch_free(hb);
        }
        if (status != M2_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != M2_OK) {
        if (best) cudaGraphExecDestroy(best);
        if (best_pipe) pipe_free(best_pipe);
        if (best_hb) hbatch_free(best_hb);
        (void)cudaGetLastError();  // reported: not again by a later launch check
        return status;
    }
    g_batch_tuning = rows;
    *out = best;
    *out_pipe = best_pipe;
    *out_hb = best_hb;
    return M2_OK;
}

}  // namespace

// Drop cached batch graphs that reference plan p (called before p is freed).
void purge_batch_graphs(const m2nufft_plan_s* p) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        const auto& k = it->key;  // [nsig, mode, plans..., buffers...]
        const int64_t n = (int64_t)k[0];
        bool hit = false;
        for (int64_t s = 0; s < n && !hit; ++s) hit = k[2 + s] == (uintptr_t)p;
        if (hit) {
            drop_entry(*it);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace m2

namespace m2 {
namespace {

// Uneven batches with or without the F-statistic outputs (Fs NULL: none); `fn` names the entry
// point in error messages.
m2_status exec_batch_impl(const m2nufft_plan_t* plans, const void* const* xs, int64_t nsig, void* const* Js,
                          void* const* Es, void* const* Ps, void* const* Fs, void* stream, const char* fn) {
    clear_error();
    if (nsig < 0 || (nsig > 0 && (!plans || !xs))) {
        set_error("%s: invalid arguments", fn);
        return M2_ERR_ARG;
    }
    if (nsig == 0) return M2_OK;
    for (int64_t s = 0; s < nsig; ++s) {
        if (!plans[s] || !xs[s]) {
            set_error("%s: plan or x %lld is NULL", fn, (long long)s);
            return M2_ERR_ARG;
        }
        if (plans[s]->precision != plans[0]->precision || plans[s]->device != plans[0]->device) {
            set_error("%s: plans differ in precision or device", fn);
            return M2_ERR_ARG;
        }
        if (Fs && Fs[s] && plans[s]->g.K < 2) {
            set_error("%s: signal %lld: the F-statistic needs K >= 2 tapers (F(2, 2K - 2))", fn, (long long)s);
            return M2_ERR_ARG;
        }
        if (Fs && Fs[s] && plans[s]->complex_taper) {
            set_error("%s: signal %lld: the F-statistic is formed for full-band plans (real tapers, f_c0 = 0)", fn,
                      (long long)s);
            return M2_ERR_ARG;
        }
    }
    bool any_f = false;
    for (int64_t s = 0; s < nsig && Fs; ++s) any_f = any_f || Fs[s];
    if (!any_f) Fs = nullptr;
    for (int64_t s = 0; s < nsig; ++s) M2_TRY(check_stage_status(plans[s]));
    const int dev = plans[0]->device;
    DeviceGuard guard(dev);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<uintptr_t> key;
    key.reserve(2 + 6 * nsig);
    const int mode = g_batch_mode.load();
    key.push_back((uintptr_t)nsig);
    key.push_back((uintptr_t)mode);
    for (int64_t s = 0; s < nsig; ++s) key.push_back((uintptr_t)plans[s]);
    for (int64_t s = 0; s < nsig; ++s) key.push_back((uintptr_t)xs[s]);
    for (int64_t s = 0; s < nsig; ++s) key.push_back((uintptr_t)(Js ? Js[s] : nullptr));
    for (int64_t s = 0; s < nsig; ++s) key.push_back((uintptr_t)(Es ? Es[s] : nullptr));
    for (int64_t s = 0; s < nsig; ++s) key.push_back((uintptr_t)(Ps ? Ps[s] : nullptr));
    for (int64_t s = 0; s < nsig; ++s) key.push_back((uintptr_t)(Fs ? Fs[s] : nullptr));

    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
        if (it->device == dev && it->key == key) {
            g_graphs.splice(g_graphs.begin(), g_graphs, it);
            if (g_graphs.front().pipe) {
                M2_TRY(pipe_check(g_graphs.front().pipe));
                pipe_batch_mark_launched(g_graphs.front().pipe);
            }
            M2_CUDA_TRY(cudaGraphLaunch(g_graphs.front().exec, st));
            return M2_OK;
        }
    }
    BatchResources* res = nullptr;
    M2_TRY(batch_resources(dev, &res));
    cudaGraphExec_t exec = nullptr;
    PipeLaunch* pipe = nullptr;
    HBatch* hb = nullptr;
    bool all_packed = plans[0]->precision == 32;
    for (int64_t s = 0; s < nsig && all_packed; ++s) all_packed = plans[s]->g.path >= 2;
    if (all_packed && mode == 2) {
        M2_TRY(tune_packed_batch(plans, xs, nsig, Js, Es, Ps, Fs, *res, st, &exec, &pipe, &hb));
    } else if (all_packed) {
        // the persistent kernel forms no F-statistic: such batches run stage-batched
        if (mode == 1 && !Fs) M2_TRY(pipe_batch_create(plans, xs, nsig, Js, Es, Ps, &pipe));
        else M2_TRY(hbatch_create(plans, xs, nsig, Js, Es, Ps, Fs, HBConfig{}, &hb));
        const m2_status cs = capture_packed_batch(pipe, hb, *res, &exec);
        if (cs != M2_OK) {
            if (pipe) pipe_free(pipe);
            if (hb) hbatch_free(hb);
            return cs;
        }
    } else {
        M2_TRY(capture_batch(plans, xs, nsig, Js, Es, Ps, Fs, *res, &exec));
    }
    g_graphs.push_front(GraphEntry{dev, std::move(key), exec, pipe, hb});
    while (g_graphs.size() > kMaxGraphs) {
        drop_entry(g_graphs.back());
        g_graphs.pop_back();
    }
    M2_CUDA_TRY(cudaGraphLaunch(exec, st));
    return M2_OK;
}

}  // namespace
}  // namespace m2

extern "C" m2_status m2nufft_exec_batch(const m2nufft_plan_t* plans, const void* const* xs, int64_t nsig,
                                        void* const* Js, void* const* Es, void* const* Ps, void* stream) {
    return m2::exec_batch_impl(plans, xs, nsig, Js, Es, Ps, nullptr, stream, "m2nufft_exec_batch");
}

extern "C" m2_status m2nufft_exec_batch_ftest(const m2nufft_plan_t* plans, const void* const* xs, int64_t nsig,
                                              void* const* Js, void* const* Es, void* const* Ps, void* const* Fs,
                                              void* stream) {
    if (!Fs) {
        m2::clear_error();
        m2::set_error("m2nufft_exec_batch_ftest: Fs is NULL");
        return M2_ERR_ARG;
    }
    return m2::exec_batch_impl(plans, xs, nsig, Js, Es, Ps, Fs, stream, "m2nufft_exec_batch_ftest");
}

extern "C" m2_status m2nufft_set_timing(m2nufft_plan_t p, int enable) {
    m2::clear_error();
    if (!p) {
        m2::set_error("plan is NULL");
        return M2_ERR_ARG;
    }
    p->timing = enable ? 1 : 0;
    return M2_OK;
}

extern "C" m2_status m2nufft_get_timing(m2nufft_plan_t p, double* ms, int64_t* launches) {
    m2::clear_error();
    if (!p) {
        m2::set_error("plan is NULL");
        return M2_ERR_ARG;
    }
    m2::DeviceGuard guard(p->device);
    for (int k = 0; k < 4; ++k) {
        auto& b = p->ev_rec[k][0];
        auto& e = p->ev_rec[k][1];
        const size_t n = std::min(b.size(), e.size());
        for (size_t i = 0; i < n; ++i) {
            float t = 0.f;
            if (cudaEventSynchronize(e[i]) == cudaSuccess && cudaEventElapsedTime(&t, b[i], e[i]) == cudaSuccess) {
                p->timing_ms[k] += t;
                p->timing_launches[k] += 1;
            }
        }
        for (cudaEvent_t ev : b) p->ev_pool.push_back(ev);
        for (cudaEvent_t ev : e) p->ev_pool.push_back(ev);
        b.clear();
        e.clear();
    }
    for (int k = 0; k < 4; ++k) {
        if (ms) ms[k] = p->timing_ms[k];
        if (launches) launches[k] = p->timing_launches[k];
        p->timing_ms[k] = 0;
        p->timing_launches[k] = 0;
    }
    return M2_OK;
}

extern "C" int m2nufft_set_batch_mode(int mode) {
    m2::clear_error();
    if (mode < 0 || mode > 2) {
        m2::set_error("m2nufft_set_batch_mode: mode must be 0, 1 or 2");
        return -1;
    }
    return m2::g_batch_mode.exchange(mode);
}

extern "C" m2_status m2nufft_get_batch_tuning(int* n, int* config, double* ms) {
    m2::clear_error();
    if (!n || *n < 0) {
        m2::set_error("m2nufft_get_batch_tuning: n must point to the capacity (>= 0)");
        return M2_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(m2::g_batch_mu);
    const int cnt = (int)m2::g_batch_tuning.size();
    const int m = std::min(*n, cnt);
    for (int i = 0; i < m; ++i) {
        const auto& r = m2::g_batch_tuning[(size_t)i];
        if (config) {
            config[4 * i + 0] = r.mode;
            config[4 * i + 1] = r.cfg.spread_tiles;
            config[4 * i + 2] = r.cfg.row_warps;
            config[4 * i + 3] = r.cfg.epi_t1;
        }
        if (ms) ms[i] = r.ms;
    }
    *n = cnt;
    return M2_OK;
}
