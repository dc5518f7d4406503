// Device-side stages of the packed FP32 exec path, shared by the four
// stand-alone kernels (fast.cu) and the persistent pipelined kernel (pipe.cu).
//
// Mathematics (Sec. 3.2, Eq. eigencoefficients and Eq.
// power_spectrum_estimator, evaluated by a type-1 nonuniform FFT):
//   * two real tapers share one complex FFT: the spread grid of taper pair j is
//     g_{2j} + i g_{2j+1}; both grids are real, so their transforms follow from
//     the packed transform Zp at k and nf - k:
//         X_{2j}[k]   = (Zp[k] + conj(Zp[nf-k])) / 2
//         X_{2j+1}[k] = (Zp[k] - conj(Zp[nf-k])) / (2i);
//   * four-step FFT nf = n1 * 1024 with the spread support in the first `rows`
//     rows: column DFTs per coset k1 = r + C q (C = n1/F) by folding the inputs
//     modulo F and one F-point register FFT, then 1024-point row FFTs in place
//     (one warp per row, 32 x 32 in registers, one padded shared-memory
//     transpose; only the in-band columns are written back);
//   * epilogue: one thread per output pair (m, -m): J(-m) = conj J(m) since
//     both tapers are real and the deconvolution factor satisfies
//     s(-m) = conj s(m); P-hat summed over the pairs in registers.  Tiles of
//     32 rows x 16 columns and their partners are staged in shared memory so
//     that both the loads and the J/E/P stores are coalesced.
// Intermediates (g, Z) are read with ld.global.cg (L2, not L1), so stages may
// consume data written by other CTAs of the same kernel.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace m2 {
namespace packed {

constexpr int kRowLen = 1024;  // n2
constexpr int kRowPad = 1060;  // per-warp transpose / row buffer: >= 32 x 33 (padded transpose)
constexpr int kColWarps = 4;   // warps per 32-column group of the column pass

struct Tw32 {
    float2 w[16];  // exp(-i 2 pi e / 32), e < 16
};

// Complex product and squared magnitude with the rounding spelled out (one product rounded, the
// other fused), so that every kernel that inlines a stage -- whatever the compiler would contract
// there -- computes the same bits.
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float norm2f(float2 a) { return __fmaf_rn(a.x, a.x, __fmul_rn(a.y, a.y)); }

__host__ __device__ constexpr int brev(int v, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
    return r;
}
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// In-register radix-2 decimation-in-frequency FFT of length N <= 32 (natural
// input, bit-reversed output): v[q] holds X[brev(q)].
template <int N>
__device__ __forceinline__ void fft_reg(float2 (&v)[N], const Tw32& tw) {
#pragma unroll
    for (int h = N / 2; h >= 1; h /= 2) {
#pragma unroll
        for (int blk = 0; blk < N; blk += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const float2 a = v[blk + j], b = v[blk + j + h];
                v[blk + j] = make_float2(a.x + b.x, a.y + b.y);
                const float2 d = make_float2(a.x - b.x, a.y - b.y);
                const int e = j * (32 / (2 * h));
                if (e == 0) v[blk + j + h] = d;
                else if (e == 8) v[blk + j + h] = make_float2(d.y, -d.x);
                else v[blk + j + h] = cmulf(d, tw.w[e]);
            }
        }
    }
}

// Plan data the stages read (one plan; device pointers).
struct __align__(16) Ctx {
    // cell-major spreading matrix (sliced ELL, see spread_ell): per 32-cell slice {first entry,
    // entries per cell}; per entry {point word, window value}; per 256-cell tile its entry and point
    // ranges and its sample run; taper pairs point-major and the points' sample indices
    const int2* ell_slice;
    const uint2* ell_e;
    const int4* ell_tile;
    const int4* ell_run;
    const float2* tap2;    // [P][Kp]
    const int32_t* pt_src; // [P]
    int ecap, pcap, ncap;  // largest staged tile: entries, points, samples (multiples of 4)
    int N, K, Kp;
    int64_t Lg;          // spread cells per pair = rows * 1024
    int rows, n1;
    int I, i_c, nf, k2max;
    int F;                 // coset FFT length of the column pass (largest power of two <= 32 dividing n1)
    int cgw;               // persistent kernel: warps per 32-column group of the column pass (1, 2 or 4)
    int cm;                // persistent kernel: column passes (8 / cgw groups of 32 columns each) per item
    const float2* tw_n1;   // [n1]
    const float2* colT;    // [F][1024]
    const float2* colB;    // [C][1024]
    const float2* colFw;   // [C][rows] fold twiddles W_n1^{(l1 r) mod n1}
    const float2* tw1024;  // [32][32]: [cc][l] = W_1024^{cc l}
    const float2* deconv;  // [I]
    const float* wsum;     // [K] W_k^0(0) = sum_n w_k(t_n) (F-statistic), or NULL
    float wq;              // sum_k W_k^0(0)^2
    int* status;           // mapped host word [flag, code, where, 0] set by a stage whose bounded wait gave up
};

// Drop a dead 128-byte line of an intermediate from L2 without writing it back (its contents
// become undefined; the next writer of the workspace overwrites it before anyone reads it).
// p: 128-byte aligned.
__device__ __forceinline__ void discard_l2(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Load of an intermediate written earlier: kStream = streaming (evict-first) for the
// stand-alone kernels, where each value is read once; otherwise L2-only (.cg), which
// is coherent with stores made by other CTAs of the same kernel.
template <bool kStream>
__device__ __forceinline__ float2 ld_inter(const float2* p) {
    if (kStream) return __ldcs(p);
    return __ldcg(p);
}

// ---------------------------------------------------------------------------
// Asynchronous bulk copies into shared memory (cp.async.bulk, the 1-D form of the tensor memory
// accelerator's copies), completed on an mbarrier, and the bounded waits on it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// makes the barrier initialisation visible to the asynchronous proxy that completes it
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this thread's earlier shared-memory accesses (generic proxy) before later bulk copies
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// L2 policy for data read once: evict first
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// dst (shared, 16-byte aligned) <- src (global, 16-byte aligned), bytes a multiple of 16, completed
// on `bar` (whose transaction count the caller raised for it)
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ long long gtimer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr long long kStageWaitNs = 2000000000LL;  // 2 s: a copy that has not landed by then never will
// Wait for the phase with this parity to complete; false if it has not within kStageWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    if (mbar_test(bar, parity)) return true;
    const long long t0 = gtimer_ns();
    while (!mbar_test(bar, parity))
        if (gtimer_ns() - t0 > kStageWaitNs) return false;
    return true;
}
// Record a stage that gave up waiting (the host reads the word at the plan's next exec).
__device__ __forceinline__ void stage_timeout(int* status, int where) {
    if (!status) return;
    if (atomicExch(status, 1) == 0) {
        status[1] = (int)M2_ERR_TIMEOUT;
        status[2] = where;
        __threadfence_system();
    }
}

// ---------------------------------------------------------------------------
// Spreading by the plan's cell-major spreading matrix (sliced ELL, slices of 32 cells):
//   g[j][c] = sum over the points p whose window covers cell c (ascending p) of
//             ((u_{2j}[p] + i u_{2j+1}[p]) * phi_p(c)) x[src(p)]
// with phi_p(c) = phi(c - u_p) the exponential-of-semicircle window.  The window values depend only
// on the sampling pattern, so the plan evaluates them once (FP64, rounded to FP32) and stores them
// per (cell, point) entry; spreading a signal is then a streaming sparse product with no
// transcendental functions.  Entry e of cell 32 s + l (slice s) is ell_e[sl.x + 32 e + l]
// (sl = ell_slice[s] = {first entry, entries per cell}): {point word, phi bits}, point word
// 0xffffffff = padding.  Per 256-cell tile, ell_tile = {first entry, entries, first point,
// points} (its slices' entries and its points are contiguous) and ell_run = {first sample,
// samples, staged, 0}.  Staged tiles (staged != 0): the point word is (p - first point) |
// (src(p) - first sample) << 16, and thread 0 copies the tile's entries, its points' taper pairs
// (tap2 [P][Kp], point-major) and the run of samples of each of the SB signals into shared memory
// with cp.async.bulk, completed on one mbarrier; the cells then read only shared memory.  Other
// tiles: the point word is p, and entries, tapers (tap2) and samples (src = pt_src[p]) are read
// from global memory.  A warp spreads one slice (lane l: cell 32 s + l), a 256-thread CTA one tile
// for nsb signals (x and g strided by N and Kp * Lg), SB at a time; each product is rounded as
//   w = phi * u (per component), acc = fma(w, x, acc)   in ascending entry order,
// so every executor writes the same bits.  A copy that has not landed within 2 s is recorded in
// c.status and the CTA writes nothing.  Called by all 256 threads of the CTA.
// smem (16-byte aligned): spread_ell_smem_bytes(Kp, nsb, ecap, pcap, ncap).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t spread_ell_tap_off(int ecap) { return 16 + (size_t)8 * ecap; }
__host__ __device__ constexpr size_t spread_ell_x_off(int Kp, int ecap, int pcap) {
    return spread_ell_tap_off(ecap) + (((size_t)8 * ((size_t)pcap * Kp + 2) + 15) & ~(size_t)15);
}
__host__ __device__ constexpr size_t spread_ell_smem_bytes(int Kp, int SB, int ecap, int pcap, int ncap) {
    return spread_ell_x_off(Kp, ecap, pcap) + (size_t)4 * SB * (ncap > 0 ? ncap + 8 : 0);
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
constexpr unsigned kEllPad = 0xffffffffu;

// the products of one entry for SB signals: w_j = phi * u_j, acc[b][j] += w_j * x_b
template <int KP, int SB>
__device__ __forceinline__ void spread_ell_mac(float2 (&acc)[SB][KP], const float2 (&u)[KP], float phi,
                                               const float (&xv)[SB], int nsb) {
#pragma unroll
    for (int j = 0; j < KP; ++j) {
        const float2 wj = make_float2(__fmul_rn(phi, u[j].x), __fmul_rn(phi, u[j].y));
#pragma unroll
        for (int b = 0; b < SB; ++b) {
            if (b < nsb) {
                acc[b][j].x = __fmaf_rn(wj.x, xv[b], acc[b][j].x);
                acc[b][j].y = __fmaf_rn(wj.y, xv[b], acc[b][j].y);
            }
        }
    }
}

template <int KP, int SB>
__device__ __forceinline__ void spread_ell(const Ctx& c, const float* __restrict__ x, int nsb, int tile,
                                           float2* __restrict__ g, unsigned char* smem) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    const uint2* s_e = reinterpret_cast<const uint2*>(smem + 16);
    const int4 tb = __ldg(c.ell_tile + tile);  // {first entry, entries, first point, points}
    const int4 tr = __ldg(c.ell_run + tile);   // {first sample, samples, staged, 0}
    const bool staged = tr.z != 0;             // uniform over the CTA
    const int Kp = c.Kp;
    const int ldx = c.ncap + 8;
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)tile * (kSpreadTile / 32) + (threadIdx.x >> 5);
    const int64_t cell = s * 32 + lane;
    const int2 sl = cell < c.Lg ? __ldg(c.ell_slice + s) : make_int2(0, 0);  // loaded while the copies fly
    const float2* s_tap = reinterpret_cast<const float2*>(smem + spread_ell_tap_off(c.ecap));
    const float* s_x = reinterpret_cast<const float*>(smem + spread_ell_x_off(Kp, c.ecap, c.pcap));
    int to = 0;  // staged: position of point tb.z's taper pairs in s_tap (float2 units)
    // staged: position of sample tr.x of signal b in s_x[b] (the copy starts on the 16-byte boundary
    // at or below it)
    auto xoff = [&](int b) { return (int)((reinterpret_cast<uintptr_t>(x + (int64_t)b * c.N + tr.x) & 15u) >> 2); };
    if (staged) {
        fence_async_smem();  // earlier reads of this shared memory before the copies overwrite it
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_init_fence();
        }
        __syncthreads();
        const uintptr_t ta = reinterpret_cast<uintptr_t>(c.tap2 + (int64_t)tb.z * Kp);
        const uintptr_t tlo = ta & ~(uintptr_t)15, thi = (ta + (uintptr_t)8 * tb.w * Kp + 15) & ~(uintptr_t)15;
        to = (int)((ta - tlo) >> 3);
        if (threadIdx.x == 0) {
            unsigned total = 8u * (unsigned)tb.y + (unsigned)(thi - tlo);
            for (int b = 0; b < nsb; ++b) {
                const uintptr_t a0 = reinterpret_cast<uintptr_t>(x + (int64_t)b * c.N + tr.x);
                total += (unsigned)(((a0 + 4u * (unsigned)tr.y + 15) & ~(uintptr_t)15) - (a0 & ~(uintptr_t)15));
            }
            const uint64_t pol = l2_evict_first_policy();
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(total)
                         : "memory");
            if (tb.y > 0) bulk_copy(smem + 16, c.ell_e + tb.x, 8u * (unsigned)tb.y, bar, pol);
            if (thi > tlo)
                bulk_copy(smem + spread_ell_tap_off(c.ecap), reinterpret_cast<const void*>(tlo), (unsigned)(thi - tlo),
                          bar, pol);
            for (int b = 0; b < nsb; ++b) {
                const uintptr_t a0 = reinterpret_cast<uintptr_t>(x + (int64_t)b * c.N + tr.x);
                const uintptr_t lo = a0 & ~(uintptr_t)15, hi = (a0 + 4u * (unsigned)tr.y + 15) & ~(uintptr_t)15;
                bulk_copy(const_cast<float*>(s_x) + b * ldx, reinterpret_cast<const void*>(lo), (unsigned)(hi - lo),
                          bar, pol);
            }
        }
        // one thread waits on the barrier (the others hold at the CTA barrier, taking no issue slots);
        // the CTA barrier then makes the copied data visible to every thread
        const bool late = threadIdx.x == 0 && !mbar_wait(bar, 0);
        const bool any_late = __syncthreads_or(late);
        if (threadIdx.x == 0 && !any_late) mbar_inval(bar);
        if (any_late) {
            if (threadIdx.x == 0) stage_timeout(c.status, tile);
            return;
        }
    }
    if (cell >= c.Lg) return;  // no barrier follows
    // with Kp == KP even, the tapers of a point are 16-byte aligned in s_tap (the copy starts on a
    // 16-byte boundary and to = 0): read them two pairs at a time
    const bool vec = (KP % 2 == 0) && Kp == KP;
    // the signals in groups of SB, each group's accumulators in registers
    for (int b0 = 0; b0 < nsb; b0 += SB) {
        const int ng = min(SB, nsb - b0);
        float2 acc[SB][KP];
#pragma unroll
        for (int b = 0; b < SB; ++b)
#pragma unroll
            for (int j = 0; j < KP; ++j) acc[b][j] = make_float2(0.f, 0.f);
        if (staged) {
            const uint2* es = s_e + (sl.x - tb.x) + lane;
            int xo[SB];
#pragma unroll
            for (int b = 0; b < SB; ++b) xo[b] = (b0 + b) * ldx + (b < ng ? xoff(b0 + b) : 0);
#pragma unroll 4
            for (int e = 0; e < sl.y; ++e) {
                const uint2 en = es[32 * e];
                if (en.x == kEllPad) continue;
                const int pl = (int)(en.x & 0xffffu), xl = (int)(en.x >> 16);
                float2 u[KP];
                if (vec) {
                    const float4* t4 = reinterpret_cast<const float4*>(s_tap + to + pl * KP);
#pragma unroll
                    for (int j = 0; j < KP / 2; ++j) {
                        const float4 v = t4[j];
                        u[2 * j] = make_float2(v.x, v.y);
                        u[2 * j + 1] = make_float2(v.z, v.w);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < KP; ++j) u[j] = j < Kp ? s_tap[to + pl * Kp + j] : make_float2(0.f, 0.f);
                }
                float xv[SB];
#pragma unroll
                for (int b = 0; b < SB; ++b) xv[b] = b < ng ? s_x[xo[b] + xl] : 0.f;
                spread_ell_mac<KP, SB>(acc, u, __uint_as_float(en.y), xv, ng);
            }
        } else {
            const uint2* eg = c.ell_e + sl.x + lane;
            const float* xg = x + (int64_t)b0 * c.N;
#pragma unroll 2
            for (int e = 0; e < sl.y; ++e) {
                const uint2 en = __ldg(eg + 32 * e);
                if (en.x == kEllPad) continue;
                const int p = (int)en.x;
                const int q = __ldg(c.pt_src + p);
                float2 u[KP];
#pragma unroll
                for (int j = 0; j < KP; ++j) u[j] = j < Kp ? __ldg(c.tap2 + (int64_t)p * Kp + j) : make_float2(0.f, 0.f);
                float xv[SB];
#pragma unroll
                for (int b = 0; b < SB; ++b) xv[b] = b < ng ? __ldg(xg + (int64_t)b * c.N + q) : 0.f;
                spread_ell_mac<KP, SB>(acc, u, __uint_as_float(en.y), xv, ng);
            }
        }
#pragma unroll
        for (int b = 0; b < SB; ++b)
            if (b < ng) {
#pragma unroll
                for (int j = 0; j < KP; ++j)
                    if (j < Kp) g[((int64_t)(b0 + b) * Kp + j) * c.Lg + cell] = acc[b][j];
            }
    }
}

// ---------------------------------------------------------------------------
// column pass for 32 columns starting at colbase, done by a group of gw warps
// (gwarp = this warp's index in the group); every warp of the CTA calls this
// once per pass, so the CTA-wide barriers line up:
//   Z[k1][l2] = W_nf^{l2 k1} sum_{l1 < rows} g[l1][l2] W_n1^{l1 k1}
// The group's warps share the C = n1 / F cosets k1 = r + C q.  Two forms with the
// same arithmetic (every product rounded as cmulf does, the fold adds in row
// order), so they write the same bits:
//   kStaged: s_tw is the fold-twiddle table [C][rows], s_tw[r][l1] =
//     W_n1^{(l1 r) mod n1} (fill_fold_twiddles), and the group's [C][32] coset
//     factors W_nf^{l2 r} are staged with its inputs, so the coset loop reads only
//     shared memory -- for CTAs with several cosets per warp;
//   otherwise: s_tw is the [n1] table W_n1^q (fill_n1_twiddles), the twiddle
//     index (l1 r) mod n1 advances by r per row and the coset factor is read in
//     the loop -- a shorter prologue, for CTAs with one coset per warp.
// The tables are filled by all threads of the CTA before the call (the first
// barrier inside publishes them).  smem: this group's [rows][32] inputs, [F][32]
// output twiddles W_nf^{l2 C q} (and with kStaged the [C][32] coset factors).
// ---------------------------------------------------------------------------
__host__ __device__ inline int cols_cosets(int n1, int F) { return n1 / F; }
// twiddle table of the CTA, float2 units
__host__ __device__ inline size_t cols_tw_f2(bool staged, int n1, int rows, int F) {
    return staged ? (size_t)cols_cosets(n1, F) * rows : (size_t)n1;
}
__device__ __forceinline__ void fill_fold_twiddles(const Ctx& c, int F, float2* s_tw) {
    const int n = cols_cosets(c.n1, F) * c.rows;
    for (int e = threadIdx.x; e < n; e += blockDim.x) s_tw[e] = __ldg(c.colFw + e);
}
__device__ __forceinline__ void fill_n1_twiddles(const Ctx& c, float2* s_tw) {
    for (int q = threadIdx.x; q < c.n1; q += blockDim.x) s_tw[q] = __ldg(c.tw_n1 + q);
}

template <int F, bool kStaged>
__device__ __forceinline__ void cols_group(const Ctx& c, const Tw32& tw, const float2* __restrict__ gj,
                                           float2* __restrict__ Zj, int colbase, int gwarp, int gw,
                                           const float2* s_tw, float2* smem) {
    const int lane = threadIdx.x & 31;
    const int l2 = colbase + lane;
    const int n1 = c.n1, rows = c.rows;
    const int C = n1 / F;
    float2* s_in = smem;                // [rows][32]
    float2* s_T = s_in + rows * 32;     // [F][32]
    float2* s_B = s_T + F * 32;         // kStaged: [C][32]
    for (int l1 = gwarp; l1 < rows; l1 += gw) s_in[l1 * 32 + lane] = __ldcg(gj + (int64_t)l1 * kRowLen + l2);
    for (int q = gwarp; q < F; q += gw) s_T[q * 32 + lane] = __ldg(c.colT + q * kRowLen + l2);
    if (kStaged)
        for (int r = gwarp; r < C; r += gw) s_B[r * 32 + lane] = __ldg(c.colB + (int64_t)r * kRowLen + l2);
    __syncthreads();
    const int nfold = (rows + F - 1) / F;
    for (int r = gwarp; r < C; r += gw) {
        const float2 base = kStaged ? s_B[r * 32 + lane] : __ldg(c.colB + (int64_t)r * kRowLen + l2);
        float2 v[F];
        int tix = 0;  // (l1 * r) mod n1, advanced incrementally (the [n1]-table form)
        // the first F rows set the fold sums (the same values as adding them to zero, up to the
        // sign of an exact zero), the later blocks of F rows add to them in row order
#pragma unroll
        for (int q = 0; q < F; ++q) {
            if (q < rows) {
                const float2 t = kStaged ? s_tw[r * rows + q] : s_tw[tix];
                v[q] = cmulf(s_in[q * 32 + lane], t);
            } else {
                v[q] = make_float2(0.f, 0.f);
            }
            if (!kStaged) {
                tix += r;
                if (tix >= n1) tix -= n1;
            }
        }
        for (int f = 1; f < nfold; ++f) {
#pragma unroll
            for (int q = 0; q < F; ++q) {
                const int l1 = f * F + q;
                if (l1 < rows) {
                    const float2 t = kStaged ? s_tw[r * rows + l1] : s_tw[tix];
                    const float2 p = cmulf(s_in[l1 * 32 + lane], t);
                    v[q].x += p.x;
                    v[q].y += p.y;
                }
                if (!kStaged) {
                    tix += r;
                    if (tix >= n1) tix -= n1;
                }
            }
        }
        fft_reg<F>(v, tw);
        float2* Zr = Zj + (int64_t)r * kRowLen + l2;
#pragma unroll
        for (int q = 0; q < F; ++q) {
            const float2 t = cmulf(base, s_T[q * 32 + lane]);
            Zr[(int64_t)(C * q) * kRowLen] = cmulf(v[brev(q, ilog2c(F))], t);
        }
    }
    __syncthreads();  // smem reuse
}

// shared memory of one column group (float2 units, excluding the CTA's twiddle table)
__host__ __device__ inline size_t cols_group_f2(bool staged, int rows, int F, int n1) {
    return (size_t)rows * 32 + (size_t)F * 32 + (staged ? (size_t)cols_cosets(n1, F) * 32 : 0);
}

// One 1024-point row FFT by one warp, in place: the in-band transforms
//   Y[k2] = sum_{l2} Zr[l2] W_1024^{l2 k2},   k2 <= k2max or k2 >= 1023 - k2max,
// overwrite Zr[k2]; the other columns keep stale values (nothing reads them).  Lane l loads and
// stores only the entries l + 32 a, so the lanes need no ordering among themselves.  Each store
// of the warp covers 32 consecutive columns (256 bytes).  S: >= 32 x 33 float2 of this warp's
// shared memory, the padded transpose between the two radix-32 passes.
template <bool kStream>
__device__ __forceinline__ void rowfft_row(const Ctx& c, const Tw32& tw, float2* __restrict__ Zr, float2* S) {
    const int lane = threadIdx.x & 31;
    float2 v[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = ld_inter<kStream>(Zr + lane + 32 * a);
    fft_reg<32>(v, tw);  // over a for column b = lane: v[q] = Y[lane][brev(q)]
    // twiddle W_1024^{lane cc} from the (L1-resident) [cc][lane] table: 256 contiguous bytes per warp
    const float2* twl = c.tw1024 + lane;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int cc = brev(q, 5);
        S[cc * 33 + lane] = cmulf(v[q], __ldg(twl + 32 * cc));
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = S[lane * 33 + a];
    __syncwarp();         // S is free again
    fft_reg<32>(v, tw);  // over b for column cc = lane: v[q] = X[lane + 32 brev(q)]
    const int nlo = c.k2max + 1;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int k2 = lane + 32 * brev(q, 5);
        if (k2 < nlo || k2 >= kRowLen - nlo) __stcg(Zr + k2, v[q]);
    }
}

// ---------------------------------------------------------------------------
// row FFTs of rows [r0, r0 + nr), nr <= R, in place (warp w < nr = row r0 + w):
//   Z[k1][k2] <- sum_{l2} Z[k1][l2] W_1024^{l2 k2} for the in-band columns.
// Called by all 32 R threads of the CTA; the warps are independent.  smem (float2): R * kRowPad.
// ---------------------------------------------------------------------------
template <int R, bool kStream>
__device__ __forceinline__ void rowfft_rows(const Ctx& c, const Tw32& tw, float2* __restrict__ Zj, int r0, int nr,
                                            float2* smem) {
    const int warp = threadIdx.x >> 5;
    if (warp < nr) rowfft_row<kStream>(c, tw, Zj + (int64_t)(r0 + warp) * kRowLen, smem + warp * kRowPad);
}

inline size_t rowfft_smem_bytes(int R) { return sizeof(float2) * (size_t)R * kRowPad; }

// ---------------------------------------------------------------------------
// epilogue tiles.  Position k = k1 + n1 k2 (k2 <= k2max, the m >= 0 side) pairs with nf - k at
// (n1 - k1, 1023 - k2), or (0, 1024 - k2) for k1 = 0, in the row transforms Y[j][k1][k2] of the
// taper pairs j.  A tile is k1 in [k1a, k1a + T1) x k2 in [k2a, k2a + 16): per pair, its T1 row
// segments and their partners' (one 128-byte line each) are staged in shared memory with
// coalesced loads (issued while the previous pair is computed, so their latency is hidden), then
// each thread unpacks, deconvolves and writes J and |J|^2 at m and -m for
// its positions -- consecutive threads take consecutive k1, so consecutive bands.  P-hat (and
// with kF Thomson's F-statistic) accumulates over the pairs in registers.
// Every in-band entry of Y is read by one position only (lower columns k2 <= k2max < 512 by
// (k1, k2); upper columns >= 512 by their partner), so with kDiscard the tile's lines are dropped
// from L2 once staged (row 0's partner columns 1024 - k2 straddle two tiles: kept).
// Yb: [Kp][n1][1024] of this signal; J, E: [K][I]; P, Fout: [I] (NULL = not wanted).
// Called by all NT threads of the CTA (NT >= 2 T1; T1 * 16 / NT positions each).
// kF (Sec. 3, Eq. f_stat): C = sum_k J_k W_k / sum_k W_k^2,
//   F = |C|^2 (K - 1) sum_k W_k^2 / sum_k |J_k - C W_k|^2, equal at m and -m.
// ---------------------------------------------------------------------------
constexpr int kEpiT2 = 16;  // k2 extent of an epilogue tile: one 128-byte line
__host__ __device__ inline int epi_tiles_k2(int k2max) { return k2max / kEpiT2 + 1; }
__host__ __device__ inline int epi_tiles(int n1, int k2max, int T1) { return (n1 + T1 - 1) / T1 * epi_tiles_k2(k2max); }
__host__ __device__ constexpr size_t epi_tile_smem_bytes(int T1) { return sizeof(float2) * 2 * T1 * (kEpiT2 + 1); }

template <int kEpiT1, int NT, bool kStream, bool kF, bool kDiscard>
__device__ __forceinline__ void epi_tile(const Ctx& c, const float2* __restrict__ Yb, int tile,
                                         float2* __restrict__ J, float* __restrict__ E, float* __restrict__ P,
                                         float* __restrict__ Fout, float2* smem) {
    constexpr int LD = kEpiT2 + 1;
    constexpr int PPT = kEpiT1 * kEpiT2 / NT;
    static_assert(PPT >= 1 && PPT * NT == kEpiT1 * kEpiT2, "tile / thread count");
    static_assert(!kF || PPT == 1, "the F-statistic keeps every J_k of one position in registers");
    float2* sA = smem;                // [T1][LD] Y[j][k1][k2]
    float2* sB = smem + kEpiT1 * LD;  // [T1][LD] the partner entries
    const int n1 = c.n1, nf = c.nf, half = nf >> 1, I = c.I, K = c.K, Kp = c.Kp;
    // consecutive tiles take consecutive k1 blocks of the same 16 columns, so the CTAs running
    // together write one contiguous stretch of bands (n1 * 16 of them) of each output plane
    const int ntk1 = (n1 + kEpiT1 - 1) / kEpiT1;
    const int k1a = (tile % ntk1) * kEpiT1, k2a = (tile / ntk1) * kEpiT2;
    const int nlo = c.k2max + 1;
    const int64_t plane = (int64_t)n1 * kRowLen;

    // this thread's positions (r, cc) = (e % T1, e / T1)
    int i1[PPT], i2[PPT];
    bool v1[PPT], v2[PPT];
    float2 sd[PPT];
    float pacc[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
        const int e = threadIdx.x + u * NT;
        const int k1 = k1a + e % kEpiT1, k2 = k2a + e / kEpiT1;
        v1[u] = v2[u] = false;
        i1[u] = i2[u] = 0;
        pacc[u] = 0.f;
        sd[u] = make_float2(0.f, 0.f);
        if (k1 < n1 && k2 < nlo) {
            const int pk1 = k1 == 0 ? 0 : n1 - k1;
            const int pk2 = k1 == 0 ? (kRowLen - k2) & (kRowLen - 1) : kRowLen - 1 - k2;
            const int kk1 = k1 + n1 * k2, kk2 = pk1 + n1 * pk2;
            i1[u] = (kk1 < half ? kk1 : kk1 - nf) + c.i_c;
            i2[u] = (kk2 < half ? kk2 : kk2 - nf) + c.i_c;
            v1[u] = (unsigned)i1[u] < (unsigned)I;
            v2[u] = (unsigned)i2[u] < (unsigned)I && kk2 != kk1;
            if (v1[u]) {
                sd[u] = __ldg(c.deconv + i1[u]);
            } else if (v2[u]) {
                sd[u] = __ldg(c.deconv + i2[u]);
                sd[u].y = -sd[u].y;
            }
        }
    }
    constexpr int kMaxPairs = kF ? (kMaxK + 1) / 2 : 1;
    float2 jk[kMaxPairs][2];  // kF: J of every taper at this position, for the residual of the line fit
    float2 csum = make_float2(0.f, 0.f);

    // the tile entries this thread stages (16 threads per 128-byte row segment, so the loads are
    // coalesced), their offsets within a plane, and the values of the next pair, loaded while the
    // current pair is computed
    bool lv[PPT];
    int la[PPT], lb[PPT];  // within a plane (n1 * 1024 < 2^31)
    float2 ra[PPT], rb[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
        const int e = threadIdx.x + u * NT;
        const int lr = e / kEpiT2, lc = e % kEpiT2;
        const int k1 = k1a + lr, k2 = k2a + lc;
        lv[u] = k1 < n1 && k2 < nlo;
        const int pk1 = k1 == 0 ? 0 : n1 - k1;
        const int pk2 = k1 == 0 ? (kRowLen - k2) & (kRowLen - 1) : kRowLen - 1 - k2;
        la[u] = k1 * kRowLen + k2;
        lb[u] = pk1 * kRowLen + pk2;
        ra[u] = rb[u] = make_float2(0.f, 0.f);
    }
    auto fetch = [&](int j) {
        const float2* Yj = Yb + (int64_t)j * plane;
#pragma unroll
        for (int u = 0; u < PPT; ++u)
            if (lv[u]) {
                ra[u] = ld_inter<kStream>(Yj + la[u]);
                rb[u] = ld_inter<kStream>(Yj + lb[u]);
            }
    };
    fetch(0);

    auto pair = [&](int j) {
        const float2* Yj = Yb + (int64_t)j * plane;
        __syncthreads();  // the previous pair's reads of the tile are done
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            const int e = threadIdx.x + u * NT;
            if (lv[u]) {
                sA[(e / kEpiT2) * LD + e % kEpiT2] = ra[u];
                sB[(e / kEpiT2) * LD + e % kEpiT2] = rb[u];
            }
        }
        __syncthreads();
        if (j + 1 < Kp) fetch(j + 1);
        if (kDiscard) {
            const int t = threadIdx.x;
            if (t < kEpiT1) {
                const int k1 = k1a + t;
                if (k1 < n1) discard_l2(Yj + (int64_t)k1 * kRowLen + k2a);
            } else if (t < 2 * kEpiT1) {
                const int k1 = k1a + t - kEpiT1;
                if (k1 < n1 && k1 > 0) discard_l2(Yj + (int64_t)(n1 - k1) * kRowLen + (kRowLen - kEpiT2 - k2a));
            }
        }
        const bool odd = 2 * j + 1 < K;
        const int64_t o0 = (int64_t)(2 * j) * I, o1 = o0 + I;
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            if (!v1[u] && !v2[u]) continue;
            const int e = threadIdx.x + u * NT;
            const float2 A = sA[(e % kEpiT1) * LD + e / kEpiT1];
            const float2 Bc = sB[(e % kEpiT1) * LD + e / kEpiT1];
            // X_even = (A + conj(B)) / 2 ; X_odd = (A - conj(B)) / (2i)
            const float2 j0 = cmulf(make_float2(0.5f * (A.x + Bc.x), 0.5f * (A.y - Bc.y)), sd[u]);
            const float p0 = norm2f(j0);
            if (J) {
                if (v1[u]) __stcs(J + o0 + i1[u], j0);
                if (v2[u]) __stcs(J + o0 + i2[u], make_float2(j0.x, -j0.y));
            }
            if (E) {
                if (v1[u]) __stcs(E + o0 + i1[u], p0);
                if (v2[u]) __stcs(E + o0 + i2[u], p0);
            }
            pacc[u] += p0;
            if (kF) {
                const float w0 = c.wsum[2 * j];
                jk[kF ? j : 0][0] = j0;
                csum.x += j0.x * w0;
                csum.y += j0.y * w0;
            }
            if (odd) {
                const float2 j1 = cmulf(make_float2(0.5f * (A.y + Bc.y), -0.5f * (A.x - Bc.x)), sd[u]);
                if (kF) {
                    const float w1 = c.wsum[2 * j + 1];
                    jk[kF ? j : 0][1] = j1;
                    csum.x += j1.x * w1;
                    csum.y += j1.y * w1;
                }
                const float p1 = norm2f(j1);
                if (J) {
                    if (v1[u]) __stcs(J + o1 + i1[u], j1);
                    if (v2[u]) __stcs(J + o1 + i2[u], make_float2(j1.x, -j1.y));
                }
                if (E) {
                    if (v1[u]) __stcs(E + o1 + i1[u], p1);
                    if (v2[u]) __stcs(E + o1 + i2[u], p1);
                }
                pacc[u] += p1;
            }
        }
    };
    if constexpr (kF) {
#pragma unroll
        for (int j = 0; j < kMaxPairs; ++j)
            if (j < Kp) pair(j);  // fully unrolled: jk stays in registers (Kp is uniform: the barriers line up)
    } else {
        for (int j = 0; j < Kp; ++j) pair(j);
    }
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
        if (P) {
            const float pv = pacc[u] * (1.0f / (float)K);
            if (v1[u]) __stcs(P + i1[u], pv);
            if (v2[u]) __stcs(P + i2[u], pv);
        }
        if (kF && Fout && (v1[u] || v2[u])) {
            const float2 ch = make_float2(csum.x / c.wq, csum.y / c.wq);  // line amplitude C at m
            float res = 0.f;
#pragma unroll
            for (int j = 0; j < kMaxPairs; ++j) {
                if (j >= Kp) break;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (2 * j + h < K) {
                        const float wk = c.wsum[2 * j + h];
                        const float rx = jk[j][h].x - ch.x * wk, ry = jk[j][h].y - ch.y * wk;
                        res += rx * rx + ry * ry;
                    }
                }
            }
            const float fv = (ch.x * ch.x + ch.y * ch.y) * (float)(K - 1) * c.wq / res;
            if (v1[u]) __stcs(Fout + i1[u], fv);
            if (v2[u]) __stcs(Fout + i2[u], fv);
        }
    }
}

// Twiddles exp(-i 2 pi e / 32), e < 16, for the register FFTs.
Tw32 make_tw32();

}  // namespace packed

// Stage context of a packed plan (host side; reads the plan's device buffers).
packed::Ctx packed_ctx(const m2nufft_plan_s* p);
// Positions on the m >= 0 side of the packed spectrum: k2 <= k2max.
int packed_k2max(const Geometry& g);

}  // namespace m2
