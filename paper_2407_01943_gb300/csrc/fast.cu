// Packed FP32 exec path (real tapers, nf = n1 * 1024, support <= 64 rows), as
// four stand-alone kernels per chunk of signals: spread, column DFTs, row FFTs,
// epilogue.  The stage bodies live in packed_stages.cuh and are shared with the
// persistent pipelined kernel (pipe.cu); see that header for the mathematics.
//
// Layout per chunk of nb signals (plan workspace):
//   g  [nb][Kp][rows * 1024]   spread grids of the taper pairs
//   Z  [nb][Kp][n1][1024]      after the column DFTs and the nf twiddle; then, in place, the
//                              row transforms (in-band columns only)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "packed_stages.cuh"

namespace m2 {

namespace packed {
Tw32 make_tw32() {
    Tw32 t;
    for (int e = 0; e < 16; ++e) {
        const double a = 2.0 * 3.141592653589793238462643383279502884 * e / 32.0;
        t.w[e] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    return t;
}
}  // namespace packed

int packed_k2max(const Geometry& g) {
    // positions k = k1 + n1 k2 on the m >= 0 side: k2 <= k2max where n1 k2 < I - i_c
    return (int)std::min<int64_t>(packed::kRowLen / 2 - 1, (g.I - g.i_c + g.n1 - 1) / g.n1);
}

packed::Ctx packed_ctx(const m2nufft_plan_s* p) {
    const Geometry& g = p->g;
    packed::Ctx c;
    c.ell_slice = p->d_ell_slice;
    c.ell_e = p->d_ell_e;
    c.ell_tile = p->d_ell_tile;
    c.ell_run = p->d_ell_run;
    c.tap2 = reinterpret_cast<const float2*>(p->d_tap2);
    c.pt_src = p->d_pt_src;
    c.ecap = p->ell_ecap;
    c.pcap = p->ell_pcap;
    c.ncap = p->ell_ncap;
    c.N = (int)g.N;
    c.K = g.K;
    c.Kp = g.kp;
    c.Lg = g.Lg;
    c.rows = (int)g.rows;
    c.n1 = (int)g.n1;
    c.I = (int)g.I;
    c.i_c = (int)g.i_c;
    c.nf = (int)g.nf;
    c.k2max = packed_k2max(g);
    c.F = g.colF;
    {
        // column items of the persistent kernel: the fewest warps per 32-column group that leave
        // each warp at most 3 of the C = n1 / F cosets and keep the groups of one pass (8 / cgw)
        // within the row stage's shared memory; then up to 4 cosets per warp per item
        const int C = (int)(g.n1 / g.colF);
        const size_t budget = packed::rowfft_smem_bytes(8);
        int gw = 4;
        for (int cand : {1, 2}) {
            const size_t sm = sizeof(float2) * (packed::cols_tw_f2(false, (int)g.n1, (int)g.rows, g.colF) +
                                                (size_t)(8 / cand) * packed::cols_group_f2(false, (int)g.rows, g.colF, (int)g.n1));
            if ((C + cand - 1) / cand <= 3 && sm <= budget) {
                gw = cand;
                break;
            }
        }
        const int cpw = (C + gw - 1) / gw;
        c.cgw = gw;
        c.cm = std::max(1, std::min(4 * gw, 4 / cpw));
    }
    c.tw_n1 = reinterpret_cast<const float2*>(p->d_twn1);
    c.colT = reinterpret_cast<const float2*>(p->d_colT);
    c.colB = reinterpret_cast<const float2*>(p->d_colB);
    c.colFw = reinterpret_cast<const float2*>(p->d_colFw);
    c.tw1024 = reinterpret_cast<const float2*>(p->d_tw1024);
    c.deconv = reinterpret_cast<const float2*>(p->d_deconv);
    c.wsum = reinterpret_cast<const float*>(p->d_wsum);
    c.wq = (float)p->wq;
    c.status = p->d_stage_status;
    return c;
}

namespace {

using packed::Ctx;
using packed::Tw32;
using packed::kColWarps;
using packed::kRowLen;

// grid (ntiles, ceil(nb / NS)): one 256-cell tile of up to NS signals per CTA, whose entries, tapers
// and sample runs are staged once; the signals are spread SB at a time (SB <= 4, or <= 2 for five
// or more taper pairs, which keeps the accumulators in registers).  Dynamic smem
// spread_ell_smem_bytes(Kp, NS, ecap, pcap, ncap).
__host__ __device__ constexpr int spread_signals(int KP) { return KP <= 4 ? 4 : 2; }
template <int KP>
__global__ void __launch_bounds__(kSpreadTile, 3) spread_ell_kernel(Ctx c, const float* __restrict__ x, int nb, int ns,
                                                                    float2* __restrict__ g) {
    extern __shared__ __align__(16) unsigned char smem_sp[];
    const int b0 = blockIdx.y * ns;
    packed::spread_ell<KP, spread_signals(KP)>(c, x + (int64_t)b0 * c.N, min(ns, nb - b0), blockIdx.x,
                                               g + (int64_t)b0 * c.Kp * c.Lg, smem_sp);
}

// Signals per CTA: as many as keep at least two CTAs per SM (and the staging within 96 KB), so a
// tile's entries and tapers are staged once for as many signals as possible (32 jitter16k signals:
// 8 per CTA, 14.3 us; one or four CTAs per SM measured 18.5 / 16.3 us).
template <int KP>
void launch_spread_packed(const Ctx& c, const float* x, int nb, float2* g, int sm_count, cudaStream_t st) {
    const int64_t ntiles = (c.Lg + kSpreadTile - 1) / kSpreadTile;
    int ns = std::max(1, nb);
    while (ns > 1 && (ntiles * ((nb + ns - 1) / ns) < 2 * (int64_t)sm_count ||
                      packed::spread_ell_smem_bytes(c.Kp, ns, c.ecap, c.pcap, c.ncap) > (size_t(96) << 10)))
        ns = (ns + 1) / 2;
    dim3 grid((unsigned)ntiles, (unsigned)((nb + ns - 1) / ns));
    spread_ell_kernel<KP><<<grid, kSpreadTile, packed::spread_ell_smem_bytes(c.Kp, ns, c.ecap, c.pcap, c.ncap), st>>>(
        c, x, nb, ns, g);
}

// grid (1024 / 32, Kp, nb): 32 columns of one taper pair per CTA of 4 warps
template <int F>
__global__ void __launch_bounds__(32 * kColWarps) cols_fast_kernel(Ctx c, Tw32 tw, const float2* __restrict__ g,
                                                                   float2* __restrict__ Z) {
    extern __shared__ float2 smem_f2[];
    float2* s_fw = smem_f2;  // [C][rows] fold twiddles
    const int j = blockIdx.y, b = blockIdx.z;
    packed::fill_fold_twiddles(c, F, s_fw);
    const int64_t pair = (int64_t)b * c.Kp + j;
    packed::cols_group<F, true>(c, tw, g + pair * c.Lg, Z + pair * (int64_t)c.n1 * kRowLen, blockIdx.x * 32,
                                threadIdx.x >> 5, kColWarps, s_fw, s_fw + packed::cols_tw_f2(true, c.n1, c.rows, F));
}

// grid (n1 / R, Kp, nb): R consecutive rows of one taper pair per CTA, one warp per row, in place;
// R = 4 at five CTAs per SM (at most 102 registers: 20 warps per SM) measured faster than R = 8 at
// two (128 registers, 16 warps)
template <int R>
__global__ void __launch_bounds__(32 * R, (R <= 4 ? 5 : 2)) rowfft_kernel(Ctx c, Tw32 tw, float2* __restrict__ Z) {
    extern __shared__ float2 smem_f2[];
    const int64_t base = ((int64_t)blockIdx.z * c.Kp + blockIdx.y) * (int64_t)c.n1 * kRowLen;
    packed::rowfft_rows<R, true>(c, tw, Z + base, blockIdx.x * R, R, smem_f2);
}

// grid (epi_tiles(n1, k2max, T1), nb): one T1 x 16 tile of positions per CTA (and its partners);
// kF adds the F-statistic output (16 x 16 tiles, 256 threads, one position each: every J_k of
// the position stays in registers; 256 threads at <= 64 registers keep four CTAs per SM).  Without
// F: three 512-thread CTAs per SM (40 registers, room for the next pair's tile values loaded while
// the current pair is computed; at four CTAs per SM the 32-register cap spills)
constexpr int kEpiT1 = 32;
constexpr int kEpiMinBlocks = 3;
__host__ __device__ constexpr int epi_t1(bool kF) { return kF ? 16 : kEpiT1; }
__host__ __device__ constexpr int epi_threads(bool kF) { return 16 * epi_t1(kF); }  // one position per thread
template <bool kF>
__global__ void __launch_bounds__(epi_threads(kF), kF ? 4 : kEpiMinBlocks) epi_kernel(Ctx c, const float2* __restrict__ Y,
                                                              float2* __restrict__ J, float* __restrict__ E,
                                                              float* __restrict__ P, float* __restrict__ F) {
    __shared__ __align__(16) float2 smem[packed::epi_tile_smem_bytes(epi_t1(kF)) / sizeof(float2)];
    const int b = blockIdx.y;
    const int64_t KI = (int64_t)c.K * c.I;
    packed::epi_tile<epi_t1(kF), epi_threads(kF), true, kF, true>(c, Y + (int64_t)b * c.Kp * c.n1 * kRowLen, blockIdx.x,
                                                     J ? J + b * KI : nullptr, E ? E + b * KI : nullptr,
                                                     P ? P + (int64_t)b * c.I : nullptr,
                                                     F ? F + (int64_t)b * c.I : nullptr, smem);
}

template <int F>
m2_status launch_cols_fast(const Ctx& c, const Tw32& tw, const float2* g, float2* Z, int nb, cudaStream_t st) {
    const size_t smem = sizeof(float2) * (packed::cols_tw_f2(true, c.n1, c.rows, F) +
                                          packed::cols_group_f2(true, c.rows, F, c.n1));
    dim3 grid((unsigned)(kRowLen / 32), (unsigned)c.Kp, (unsigned)nb);
    cols_fast_kernel<F><<<grid, 32 * kColWarps, smem, st>>>(c, tw, g, Z);
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

template <int R>
m2_status launch_rowfft(const Ctx& c, const Tw32& tw, float2* Z, int nb, cudaStream_t st) {
    dim3 grid((unsigned)(c.n1 / R), (unsigned)c.Kp, (unsigned)nb);
    rowfft_kernel<R><<<grid, 32 * R, packed::rowfft_smem_bytes(R), st>>>(c, tw, Z);
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

}  // namespace

m2_status init_fast_kernels(int smem_optin) {
    const void* spread[] = {(const void*)spread_ell_kernel<2>, (const void*)spread_ell_kernel<4>,
                            (const void*)spread_ell_kernel<8>};
    for (const void* f : spread)
        M2_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin));
    const void* funcs[] = {
        (const void*)cols_fast_kernel<2>,  (const void*)cols_fast_kernel<4>, (const void*)cols_fast_kernel<8>,
        (const void*)cols_fast_kernel<16>, (const void*)cols_fast_kernel<32>, (const void*)rowfft_kernel<2>,
        (const void*)rowfft_kernel<4>,
    };
    for (const void* f : funcs)
        M2_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin));
    return M2_OK;
}

m2_status spread_fast(m2nufft_plan_s* p, const float* x, int nb, float2* g_out, cudaStream_t st) {
    const Geometry& g = p->g;
    const Ctx c = packed_ctx(p);
    if (g.kp <= 2) launch_spread_packed<2>(c, x, nb, g_out, p->sm_count, st);
    else if (g.kp <= 4) launch_spread_packed<4>(c, x, nb, g_out, p->sm_count, st);
    else launch_spread_packed<8>(c, x, nb, g_out, p->sm_count, st);
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

m2_status exec_fast_chunk(m2nufft_plan_s* p, const float* x, int nb, float2* J, float* E, float* P, float* F,
                          cudaStream_t st, int lane, const float2* g_pre) {
    const Geometry& g = p->g;
    static const Tw32 tw = packed::make_tw32();
    const Ctx c = packed_ctx(p);
    // workspace of lane 0 (the plan's) or of lane L > 0 (for overlapped chunks)
    float2* dg = reinterpret_cast<float2*>(lane ? p->lane_g[lane] : p->d_g);
    float2* dZ = reinterpret_cast<float2*>(lane ? p->lane_Z[lane] : p->d_Z);
    if (g_pre) dg = const_cast<float2*>(g_pre);  // spread grids made beforehand for the whole exec

    if (!g_pre) {
    mark(p, 0, 0, st);
    {
        if (g.kp <= 2) launch_spread_packed<2>(c, x, nb, dg, p->sm_count, st);
        else if (g.kp <= 4) launch_spread_packed<4>(c, x, nb, dg, p->sm_count, st);
        else launch_spread_packed<8>(c, x, nb, dg, p->sm_count, st);
        M2_CUDA_TRY(cudaGetLastError());
    }
    mark(p, 0, 1, st);
    }

    mark(p, 1, 0, st);
    switch (g.colF) {
        case 2: M2_TRY(launch_cols_fast<2>(c, tw, dg, dZ, nb, st)); break;
        case 4: M2_TRY(launch_cols_fast<4>(c, tw, dg, dZ, nb, st)); break;
        case 8: M2_TRY(launch_cols_fast<8>(c, tw, dg, dZ, nb, st)); break;
        case 16: M2_TRY(launch_cols_fast<16>(c, tw, dg, dZ, nb, st)); break;
        default: M2_TRY(launch_cols_fast<32>(c, tw, dg, dZ, nb, st)); break;
    }
    mark(p, 1, 1, st);

    mark(p, 2, 0, st);
    {
        int R = 1;  // rows per CTA: largest power of two <= 4 dividing n1
        while (R < 4 && g.n1 % (R * 2) == 0) R *= 2;
        if (R == 4) M2_TRY(launch_rowfft<4>(c, tw, dZ, nb, st));
        else M2_TRY(launch_rowfft<2>(c, tw, dZ, nb, st));
    }
    mark(p, 2, 1, st);

    mark(p, 3, 0, st);
    {
        if (F) {
            dim3 grid((unsigned)packed::epi_tiles(c.n1, c.k2max, epi_t1(true)), (unsigned)nb);
            epi_kernel<true><<<grid, epi_threads(true), 0, st>>>(c, dZ, J, E, P, F);
        } else {
            dim3 grid((unsigned)packed::epi_tiles(c.n1, c.k2max, epi_t1(false)), (unsigned)nb);
            epi_kernel<false><<<grid, epi_threads(false), 0, st>>>(c, dZ, J, E, P, nullptr);
        }
        M2_CUDA_TRY(cudaGetLastError());
    }
    mark(p, 3, 1, st);
    return M2_OK;
}

}  // namespace m2
