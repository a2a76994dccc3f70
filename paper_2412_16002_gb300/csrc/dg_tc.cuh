// dg_tc.cuh -- inner stages of the split-precision path on the fifth-generation tensor
// cores (2D Euler, Q^3, tableaux whose A has only a sub-diagonal, as eq. cRKDG2-4).
//
// Every linear map of an inner stage is a small dense matrix applied to each cell's
// nodal data, the same matrix for every cell: batched over a tile of 128 cells it is a
// GEMM with M = 128 (one tensor-memory lane per cell) and one product per component:
//   evaluation map E (K = 16 nodes -> N = 48): the 16 face-point traces (Sec. 2.1), the
//     24 points of S_K (Prop. 2.2, Fig. 1) and the Gauss-weighted mean of the deviations;
//   G map (K = 48: x-fluxes and y-fluxes at the nodes, normal fluxes at the face points
//     -> N = 32): the deviation part of G = -div^loc f (the volume term with the
//     derivative matrix, minus the lifted interior-trace fluxes, eq. Gbar's edge form,
//     with the cell mean projected out), and its average as the weighted sum of the
//     face fluxes (eq. Gbar).
// Both run as tcgen05.mma kind::tf32 with the three-product split A_hi B_hi + A_hi B_lo
// + A_lo B_hi (FP32-level accuracy), A written by the threads into tensor memory with
// tcgen05.st (one lane per cell, no shared-memory staging), B (the maps, built by each
// CTA from the nodal tables and the cell sizes) in shared memory, FP32 accumulators in
// tensor memory read back with tcgen05.ld.  The pointwise work (fluxes, the limiter's
// screen and theta) stays on the CUDA cores; what k_inner_x keeps in FP64 (the stage
// averages, the averages' admissibility test, theta where the FP32 screen cannot clear a
// cell) stays FP64 here.
//
// Layout: a persistent CTA of 512 threads walks 128-cell tiles; threads t, t + 128,
// t + 256 and t + 384 share cell t (warps w, w + 4, w + 8, w + 12 address the same
// tensor-memory lanes), the r-th of them owning node row r, face r's points and S_K points
// 6r .. 6r + 5.  Per-cell reductions of the limiter combine the four threads through shared
// memory.  Tensor-memory columns (512, one CTA per SM):
//   [0, 192)    D_E, 48 per component (then A_G of components 2 and 3)
//   [192, 320)  A_E, hi and lo per component (then D_G, 32 per component)
//   [320, 512)  A_G of components 0 and 1, hi and lo
#pragma once

#include "dg_mixed.cuh"

namespace crkdg {
namespace tc {

constexpr int TM = 128;              // cells per tile
constexpr int NT = 512;              // threads per CTA (four per cell)
constexpr int QN = 4, QS = 6;        // nodes (and face points), S_K points per thread
constexpr int N = 4, NN = 16, NTR = 16, NSK = 24, M = 4;
constexpr int KE = 16, NE = 48;      // evaluation map: K, N
constexpr int KG = 48, NG = 32;      // G map: K, N
constexpr int COL_TR = 0, COL_SK = NTR, COL_MEAN = NTR + NSK;  // columns of E's outputs
constexpr int COL_GD = 0, COL_GB = NN;                          // columns of G's outputs
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t DE = 0, AE = 192, DG = 192;
__host__ __device__ constexpr uint32_t ag_col(int c) { return c < 2 ? 320 + c * 2 * KG : (c - 2) * 2 * KG; }
static_assert(DE + M * NE <= AE && AE + M * 2 * KE <= 320 && DG + M * NG <= 320, "tensor-memory plan");
static_assert(ag_col(1) + 2 * KG <= TMEM_COLS && ag_col(3) + 2 * KG <= DE + M * NE, "tensor-memory plan");

// B operands (N rows x K, K-major core matrices, no swizzle), hi and lo
constexpr int SZ_BE = NE * KE * 4, SZ_BG = NG * KG * 4;
constexpr uint32_t LBO_E = (NE / 8) * 128, LBO_G = (NG / 8) * 128, SBO = 128;
__host__ __device__ constexpr uint32_t idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ int core_off(int row, int k, int rows) {
    return (((k >> 2) * (rows >> 3) + (row >> 3)) << 7) + ((row & 7) << 4) + ((k & 3) << 2);
}
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// x rounded to TF32 (10 mantissa bits), to nearest with ties away from zero: half a TF32
// unit added to the magnitude bits (a carry into the exponent is the correct rounding up),
// then the 13 low bits cleared.  Two integer operations; equal to cvt.rna.tf32.f32 for every
// finite or infinite x.
__device__ __forceinline__ float tf32r(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
// x = hi + lo with hi its TF32 rounding; lo = x - hi is exact in FP32 and goes to the tensor
// cores as it is: they read its leading TF32 bits, so hi + lo as read is x to within 2^-21 |x|
// (|lo| <= 2^-11 |x|, and lo loses below 2^-10 |lo|), the A side of the three-product split.
__device__ __forceinline__ void split(float x, float &hi, float &lo) {
    hi = tf32r(x);
    lo = x - hi;
}
// the same with lo rounded to TF32 as well (2^-22 |x|), for the maps, built once per CTA
__device__ __forceinline__ void split_r(float x, float &hi, float &lo) {
    hi = tf32r(x);
    lo = tf32r(x - hi);
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo) {
    return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((SBO >> 4) & 0x3fffu) << 32) | (1ull << 46);
}
// D (tensor memory) += A (tensor memory) x B (shared memory)
__device__ __forceinline__ void mma(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ bool try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait (1 s) for phase `parity` of the MMA mbarrier.
__device__ __forceinline__ bool wait_mma(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = gtime();
    while (!try_wait(mbar, parity))
        if (gtime() - t0 > 1000000000ull) return false;
    return true;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void st8(uint32_t taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void st4(uint32_t taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3]))
                 : "memory");
}
__device__ __forceinline__ void ld2(uint32_t taddr, float *v) {
    uint32_t r[2];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
    v[0] = __uint_as_float(r[0]);
    v[1] = __uint_as_float(r[1]);
}
__device__ __forceinline__ void ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld4(uint32_t taddr, float *v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld1(uint32_t taddr, float &v) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    v = __uint_as_float(r);
}

// Asynchronous global -> shared copies of a tile's u^n (cp.async, one thread's own words).
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Entries of the maps (FP64, from the nodal tables and the cell sizes).
// E[o][q]: output o of the evaluation map from node q = b*n + a.
__device__ inline double map_E(const NodalTables &T, int o, int q) {
    const int a = q % N, b = q / N;
    if (o < NTR) {  // trace at face point o
        const int face = o / N, pos = o % N;
        if (face < 2) return b == pos ? (face == 0 ? T.lm[a] : T.lp[a]) : 0.0;
        return a == pos ? (face == 2 ? T.lm[b] : T.lp[b]) : 0.0;
    }
    if (o < NTR + NSK) {  // S_K point: Gauss row x Gauss--Lobatto, then Gauss--Lobatto x Gauss column
        constexpr int L = nlob(N);
        const int p = o - NTR;
        if (p < N * L) {
            const int beta = p / L, al = p % L;
            return b == beta ? T.Igl[al][a] : 0.0;
        }
        const int r = p - N * L, beta = r / L, al = r % L;
        return a == beta ? T.Igl[al][b] : 0.0;
    }
    if (o == COL_MEAN) return T.w2[q];
    return 0.0;
}
// G32[q][k]: node q of the FP32 operator from input k (x-flux at node k, y-flux at node k - NN,
// normal flux at face point k - 2 NN), before the mean is projected out.
__device__ inline double map_G32(const NodalTables &T, double rhx, double rhy, int q, int k) {
    const int a = q % N, b = q / N;
    if (k < NN) {
        const int qa = k % N, qb = k / N;
        return qb == b ? rhx * T.Dhat[a][qa] : 0.0;
    }
    if (k < 2 * NN) {
        const int kk = k - NN, ra = kk % N, rb = kk / N;
        return ra == a ? rhy * T.Dhat[b][rb] : 0.0;
    }
    const int fp = k - 2 * NN, face = fp / N, pos = fp % N;
    switch (face) {
    case 0: return pos == b ? rhx * T.liftm[a] : 0.0;
    case 1: return pos == b ? -rhx * T.liftp[a] : 0.0;
    case 2: return pos == a ? rhy * T.liftm[b] : 0.0;
    default: return pos == a ? -rhy * T.liftp[b] : 0.0;
    }
}

struct Smem {
    alignas(128) float be[2][NE * KE];   // evaluation map, hi / lo
    alignas(128) float bg[2][NG * KG];   // G map, hi / lo
    float dv0[2][QN][M][QN][TM];         // u^n deviations of the tile and of the next one (prefetched),
                                         // [buffer][row][comp][node][cell]
    alignas(8) double ub0[2][M][TM];     // u^n averages of the tile and of the next one
    alignas(8) double ubd[M][TM];        // the stage averages (FP64), one thread per cell writes them
    float ubf[M][TM];                    // their FP32 copies
    alignas(8) double red[QN][TM];       // reductions over the four threads of a cell
    int flg[QN][TM];
    unsigned long long mbar;
    uint32_t tmem;
    int fault;
};

// The four threads of a cell combine a value through shared memory (block collectives).
__device__ __forceinline__ int quad_or(Smem &S, int r, int lc, int v) {
    S.flg[r][lc] = v;
    __syncthreads();
    const int o = S.flg[0][lc] | S.flg[1][lc] | S.flg[2][lc] | S.flg[3][lc];
    __syncthreads();
    return o;
}
// double minima over the four threads (NaN propagated as -inf by the callers)
__device__ __forceinline__ double quad_mind(Smem &S, int r, int lc, double v) {
    S.red[r][lc] = v;
    __syncthreads();
    const double o = fmin(fmin(S.red[0][lc], S.red[1][lc]), fmin(S.red[2][lc], S.red[3][lc]));
    __syncthreads();
    return o;
}

}  // namespace tc

// One-time set-up of a CTA: the two maps, split, into shared memory.
__device__ inline void tc_build_maps(const Params &P, tc::Smem &S) {
    using namespace tc;
    const NodalTables &T = c_tab[N - 2];
    for (int e = threadIdx.x; e < NE * KE; e += NT) {
        const int o = e / KE, q = e % KE;
        const float v = (float)map_E(T, o, q);
        float hi, lo;
        split_r(v, hi, lo);
        const int off = core_off(o, q, NE) >> 2;
        S.be[0][off] = hi;
        S.be[1][off] = lo;
    }
    for (int e = threadIdx.x; e < NG * KG; e += NT) {
        const int o = e / KG, k = e % KG;
        double v = 0.0;
        if (o < NN) {  // deviation: G32 minus its Gauss-weighted mean over the nodes
            double mean = 0.0;
            for (int q = 0; q < NN; ++q) mean += T.w2[q] * map_G32(T, P.rhx, P.rhy, q, k);
            v = map_G32(T, P.rhx, P.rhy, o, k) - mean;
        } else if (o == COL_GB && k >= 2 * NN) {  // average: the weighted face-flux sum (eq. Gbar)
            const int fp = k - 2 * NN, face = fp / N, pos = fp % N;
            v = (float)(((face & 1) ? -0.5 : 0.5) * T.w1[pos] * (face < 2 ? P.rhx : P.rhy));
        }
        float hi, lo;
        split_r((float)v, hi, lo);
        const int off = core_off(o, k, NG) >> 2;
        S.bg[0][off] = hi;
        S.bg[1][off] = lo;
    }
}

// Inner stages of the split representation on the tensor cores (see the file header).
template <int PHYS>
__global__ void __launch_bounds__(tc::NT, 1) k_inner_tc(Params P, MixBufs X) {
    using namespace tc;
    static_assert(PHYS == PH_EULER, "the tensor-core inner stages are built for the Euler equations");
    constexpr int DIM = 2;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    tc::Smem &S = *reinterpret_cast<tc::Smem *>(tc_smem);
    const int t = threadIdx.x, w = t >> 5, lc = t & (TM - 1), r = t >> 7;  // r: node row / face
    const uint32_t lane = (uint32_t)((w & 3) * 32) << 16;
    Bufs B;
    memset(&B, 0, sizeof(B));
    B.flag = X.flag;
    B.nlim = X.nlim;
    B.thmin = X.thmin;
    tc_build_maps(P, S);
    const uint32_t mbar = saddr(&S.mbar);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.fault = 0;
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&S.tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the maps, for the tensor cores
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tm = S.tmem;
    const uint32_t be_hi = saddr(S.be[0]), be_lo = saddr(S.be[1]);
    const uint32_t bg_hi = saddr(S.bg[0]), bg_lo = saddr(S.bg[1]);
    uint32_t phase = 0;
    bool fault = false;
    const int ntiles = (P.ncell + TM - 1) / TM;
    const int dir = r >> 1;  // face r's normal direction

    // u^n of a tile into buffer b: this thread's node row of deviations, and (first thread of
    // a cell) the averages; cells past the mesh are left to the benign state set at use
    auto prefetch = [&](int tl, int b) {
        const int cl = tl * TM + lc;
        if (cl < P.ncell) {
#pragma unroll
            for (int c = 0; c < M; ++c) {
                const float *src = X.dv + ((size_t)c * P.ncell + cl) * NN + QN * r;
#pragma unroll
                for (int q = 0; q < QN; ++q) cp_async4(&S.dv0[b][r][c][q][lc], src + q);
                if (r == 0) cp_async8(&S.ub0[b][c][lc], X.ub + (size_t)c * P.ncell + cl);
            }
        }
        cp_async_commit();
    };
    int buf = 0;
    if ((int)blockIdx.x < ntiles) prefetch(blockIdx.x, 0);

    for (int tile = blockIdx.x; tile < ntiles && !fault; tile += gridDim.x, buf ^= 1) {
        const int cell = tile * TM + lc;
        const bool active = cell < P.ncell;
        const bool own = active && owned(P, cell);
        // u^n of this tile (prefetched), then the next tile's into the other buffer
        cp_async_wait_all();
        if (!active) {  // a benign admissible state for the padding cells of the last tile
#pragma unroll
            for (int c = 0; c < M; ++c) {
                if (r == 0) S.ub0[buf][c][lc] = (c == 0 || c == M - 1) ? 1.0 : 0.0;
#pragma unroll
                for (int q = 0; q < QN; ++q) S.dv0[buf][r][c][q][lc] = 0.0f;
            }
        }
        float dvc[M][QN], dacc[M][QN];
#pragma unroll
        for (int c = 0; c < M; ++c)
#pragma unroll
            for (int q = 0; q < QN; ++q) dvc[c][q] = dacc[c][q] = S.dv0[buf][r][c][q][lc];
        if (tile + (int)gridDim.x < ntiles) prefetch(tile + gridDim.x, buf ^ 1);
        float gbh[M];  // FP32 average of the previous stage's G
#pragma unroll
        for (int c = 0; c < M; ++c) gbh[c] = 0.0f;

        for (int i = 0; i < P.s && i < MAXS; ++i) {
            // stage averages (FP64 plus the FP32 increment), by the cell's first thread
            const float a_prev = i > 0 ? P.f.dtA[i][i - 1] : 0.0f;
            if (r == 0)
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const double v = i > 0 ? S.ub0[buf][c][lc] + (double)(a_prev * gbh[c]) : S.ub0[buf][c][lc];
                    S.ubd[c][lc] = v;
                    S.ubf[c][lc] = (float)v;
                }
            // ---- A_E: the deviations, split
            __syncthreads();  // the previous stage's D_G (same columns) has been read by every thread;
                              // the stage averages are in shared memory
            float ubf[M];
#pragma unroll
            for (int c = 0; c < M; ++c) ubf[c] = S.ubf[c][lc];
#pragma unroll
            for (int c = 0; c < M; ++c) {
                float hi[QN], lo[QN];
#pragma unroll
                for (int q = 0; q < QN; ++q) split(dvc[c][q], hi[q], lo[q]);
                st4(tm + lane + AE + c * 2 * KE + QN * r, hi);
                st4(tm + lane + AE + c * 2 * KE + KE + QN * r, lo);
            }
            wait_st();
            fence_before();
            __syncthreads();
            fence_after();
            if (t == 0) {
                const uint32_t id = idesc(NE);
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const uint32_t d = tm + DE + c * NE, ah = tm + AE + c * 2 * KE, al = ah + KE;
#pragma unroll
                    for (int s = 0; s < KE / 8; ++s) {
                        const uint32_t ob = 2 * s * LBO_E;
                        mma(d, ah + 8 * s, sdesc(be_hi + ob, LBO_E), id, s > 0);
                        mma(d, ah + 8 * s, sdesc(be_lo + ob, LBO_E), id, 1);
                        mma(d, al + 8 * s, sdesc(be_hi + ob, LBO_E), id, 1);
                    }
                }
                commit(mbar);
            }
            bool ok = wait_mma(mbar, phase);
            phase ^= 1u;
            fence_after();
            if (__syncthreads_or(!ok)) {
                fault = true;
                break;
            }
            // ---- read E's outputs: mean, this thread's S_K points and face-point traces
            float mean[M], sk[M][QS], tr[M][QN];
#pragma unroll
            for (int c = 0; c < M; ++c) {
                const uint32_t base = tm + lane + DE + c * NE;
                ld4(base + COL_TR + QN * r, tr[c]);
                ld4(base + COL_SK + QS * r, sk[c]);
                ld2(base + COL_SK + QS * r + 4, sk[c] + 4);
                ld1(base + COL_MEAN, mean[c]);
            }
            wait_ld();
            // ---- scaling limiter of the stage value (stages 2..s)
            float s0 = 1.0f, s1 = 1.0f;
            bool limited = false;
            if (i > 0) {
                int unsafe = 0;
#pragma unroll
                for (int j = 0; j < QS; ++j) {
                    float v[M];
#pragma unroll
                    for (int c = 0; c < M; ++c) v[c] = ubf[c] + (sk[c][j] - mean[c]);
                    if (!screen_ok<PHYS, DIM>(P, v, ubf)) unsafe = 1;
                }
                if (r == 0 && own && !screen_ok<PHYS, DIM>(P, ubf, ubf)) {
                    double ubd[M];
#pragma unroll
                    for (int c = 0; c < M; ++c) ubd[c] = S.ubd[c][lc];
                    if (!admissible<PHYS, DIM>(P, ubd)) atomicOr(B.flag, 1);
                }
                if (__syncthreads_or(unsafe)) {
                    unsafe = quad_or(S, r, lc, unsafe);  // the cell's decision
                    double ubd[M];
#pragma unroll
                    for (int c = 0; c < M; ++c) ubd[c] = S.ubd[c][lc];
                    // FP64 theta for the cells the screen could not clear
                    double mn = INFINITY;
                    if (unsafe) {
#pragma unroll
                        for (int j = 0; j < QS; ++j) {
                            const double v0 = ubd[0] + (double)(sk[0][j] - mean[0]);
                            mn = (v0 == v0) ? fmin(mn, v0) : -INFINITY;
                        }
                    }
                    mn = quad_mind(S, r, lc, mn);
                    double th1 = 1.0;
                    if (unsafe && mn < P.eps) th1 = ratio01(ubd[0] - P.eps, ubd[0] - mn);
                    if (th1 < 1.0) th1 *= kMargin;
                    double mre = INFINITY;
                    if (unsafe) {
#pragma unroll
                        for (int j = 0; j < QS; ++j) {
                            double v[M];
#pragma unroll
                            for (int c = 0; c < M; ++c) v[c] = ubd[c] + (double)(sk[c][j] - mean[c]);
                            if (th1 < 1.0) v[0] = th1 * (v[0] - ubd[0]) + ubd[0];
                            const double re = rho_e<DIM>(v);
                            mre = (re == re) ? fmin(mre, re) : -INFINITY;
                        }
                    }
                    mre = quad_mind(S, r, lc, mre);
                    double th2 = 1.0;
                    if (unsafe && !(mre >= P.eps)) {
                        const double reb = rho_e<DIM>(ubd);
                        th2 = ratio01(reb - P.eps, reb - mre) * kMargin;
                    }
                    limited = unsafe && (th1 < 1.0 || th2 < 1.0);
                    // rescale towards the average; verify on this stage's S_K evaluation
                    double tfin = th2;
#pragma unroll 1
                    for (int attempt = 0; attempt <= 4; ++attempt) {
                        s0 = limited ? (float)(th1 * tfin) : 1.0f;
                        s1 = limited ? (float)tfin : 1.0f;
                        int viol = 0;
                        if (limited) {
#pragma unroll
                            for (int j = 0; j < QS; ++j) {
                                double v[M];
#pragma unroll
                                for (int c = 0; c < M; ++c)
                                    v[c] = ubd[c] + (double)((c == 0 ? s0 : s1) * (sk[c][j] - mean[c]));
                                if (!point_ok<PHYS, DIM>(P, v)) viol = 1;
                            }
                        }
                        viol = quad_or(S, r, lc, viol);
                        if (!__syncthreads_or(viol) || attempt == 4) break;
                        if (viol) tfin = th2 * retry_factor(attempt + 1);
                    }
                    if (limited && r == 0 && own) {
                        const double trf = fmin(th1, tfin);
                        atomicAdd(B.nlim, 1ull);
                        atomicMin(B.thmin, dbits(trf > 0.0 ? trf : 0.0));
                    }
                }
            }
            // limited deviations and traces of the stage value
            if (limited) {
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const float sc = c == 0 ? s0 : s1;
#pragma unroll
                    for (int q = 0; q < QN; ++q) {
                        dvc[c][q] = sc * (dvc[c][q] - mean[c]);
                        tr[c][q] = sc * (tr[c][q] - mean[c]);
                    }
                }
            }
            // near vacuum (rho_ill) a density is taken rounded from its FP64 value, not the FP32
            // sum: at the face points (S_K points, so >= eps in the FP64 evaluation after
            // limiting) and at the nodes, so 1 / rho is that of the FP64 evaluation.  The test is
            // FP32; the FP64 repair runs behind a warp vote, so it costs nothing where no lane
            // needs it (the FP64 units are a small fraction of the FP32 ones).
            float rn[QN], td[QN];  // node densities; the face points' density deviations
            int ill = 0;
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                td[q] = tr[0][q];
#pragma unroll
                for (int c = 0; c < M; ++c) tr[c][q] += ubf[c];
                if (rho_ill(tr[0][q], ubf[0], td[q])) ill |= 1 << q;
                rn[q] = ubf[0] + dvc[0][q];
                if (rho_ill(rn[q], ubf[0], dvc[0][q])) ill |= 16 << q;
            }
            if (__any_sync(0xffffffffu, ill != 0)) {
                const double u0 = S.ubd[0][lc];
#pragma unroll
                for (int q = 0; q < QN; ++q) {
                    if (ill & (1 << q)) tr[0][q] = (float)(u0 + (double)td[q]);
                    if (ill & (16 << q)) rn[q] = (float)(u0 + (double)dvc[0][q]);
                }
            }
            // traced stages: traces and averages for the final stage
            if (P.slot[i] >= 0 && active) {
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    *reinterpret_cast<float4 *>(X.tr + ((size_t)P.slot[i] * M * P.ncell + (size_t)c * P.ncell + cell) * NTR +
                                                QN * r) = make_float4(tr[c][0], tr[c][1], tr[c][2], tr[c][3]);
                    if (r == 0) X.tavg[((size_t)P.slot[i] * M + c) * P.ncell + cell] = ubf[c];
                }
            }
            __syncthreads();  // every thread has read D_E: A_G of components 2, 3 overwrites it
            // ---- A_G: x- and y-fluxes at this thread's nodes, normal fluxes at its face points
            {
                float fx[M][QN], fy[M][QN];
#pragma unroll
                for (int q = 0; q < QN; ++q) {
                    float u[M], gx[M], gy[M];
#pragma unroll
                    for (int c = 1; c < M; ++c) u[c] = ubf[c] + dvc[c][q];
                    u[0] = rn[q];
                    flux_xy_f<PHYS>(P, u, gx, gy);
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        fx[c][q] = gx[c];
                        fy[c][q] = gy[c];
                    }
                }
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    float hi[QN], lo[QN];
                    const uint32_t ag = tm + lane + ag_col(c);
#pragma unroll
                    for (int q = 0; q < QN; ++q) split(fx[c][q], hi[q], lo[q]);
                    st4(ag + QN * r, hi);
                    st4(ag + KG + QN * r, lo);
#pragma unroll
                    for (int q = 0; q < QN; ++q) split(fy[c][q], hi[q], lo[q]);
                    st4(ag + NN + QN * r, hi);
                    st4(ag + KG + NN + QN * r, lo);
                }
            }
            {
                float tf[M][QN];
#pragma unroll
                for (int j = 0; j < QN; ++j) {
                    float u[M], f[M];
#pragma unroll
                    for (int c = 0; c < M; ++c) u[c] = tr[c][j];
                    flux_dir_f<PHYS, DIM>(P, u, dir, f);
#pragma unroll
                    for (int c = 0; c < M; ++c) tf[c][j] = f[c];
                }
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    float hi[QN], lo[QN];
                    const uint32_t ag = tm + lane + ag_col(c);
#pragma unroll
                    for (int q = 0; q < QN; ++q) split(tf[c][q], hi[q], lo[q]);
                    st4(ag + 2 * NN + QN * r, hi);
                    st4(ag + KG + 2 * NN + QN * r, lo);
                }
            }
            wait_st();
            fence_before();
            __syncthreads();
            fence_after();
            if (t == 0) {
                const uint32_t id = idesc(NG);
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const uint32_t d = tm + DG + c * NG, ah = tm + ag_col(c), al = ah + KG;
#pragma unroll
                    for (int s = 0; s < KG / 8; ++s) {
                        const uint32_t ob = 2 * s * LBO_G;
                        mma(d, ah + 8 * s, sdesc(bg_hi + ob, LBO_G), id, s > 0);
                        mma(d, ah + 8 * s, sdesc(bg_lo + ob, LBO_G), id, 1);
                        mma(d, al + 8 * s, sdesc(bg_hi + ob, LBO_G), id, 1);
                    }
                }
                commit(mbar);
            }
            ok = wait_mma(mbar, phase);
            phase ^= 1u;
            fence_after();
            if (__syncthreads_or(!ok)) {
                fault = true;
                break;
            }
            // ---- G: deviations at this thread's nodes and the cell average
            const float b_i = P.f.dtb[i];
            const float a_next = i + 1 < P.s ? P.f.dtA[i + 1][i] : 0.0f;
            float gd[M][QN];
#pragma unroll
            for (int c = 0; c < M; ++c) {
                ld4(tm + lane + DG + c * NG + COL_GD + QN * r, gd[c]);
                ld1(tm + lane + DG + c * NG + COL_GB, gbh[c]);
            }
            wait_ld();
#pragma unroll
            for (int c = 0; c < M; ++c)
#pragma unroll
                for (int q = 0; q < QN; ++q) {
                    if (b_i != 0.0f) dacc[c][q] = fmaf(b_i, gd[c][q], dacc[c][q]);
                    dvc[c][q] = fmaf(a_next, gd[c][q], S.dv0[buf][r][c][q][lc]);
                }
        }
        if (fault) break;
        if (active) {
#pragma unroll
            for (int c = 0; c < M; ++c)
                *reinterpret_cast<float4 *>(X.dv_s + ((size_t)c * P.ncell + cell) * NN + QN * r) =
                    make_float4(dacc[c][0], dacc[c][1], dacc[c][2], dacc[c][3]);
        }
    }
    cp_async_wait_all();  // no copy into this CTA's shared memory outlives it
    if (fault && t == 0) {
        atomicOr(X.flag, 2);  // the host reports CRKDG_E_TIMEOUT
        // an MMA group that never signalled: wait (bounded) once more before the memory goes
        wait_mma(mbar, phase ^ 1u);
    }
    fence_before();
    __syncthreads();
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TMEM_COLS) : "memory");
}

}  // namespace crkdg

namespace crkdg {

// Host launcher: one persistent CTA per SM (the kernel holds all 512 tensor-memory columns).
inline cudaError_t launch_inner_tc(cudaStream_t st, const Params &P, const MixBufs &X) {
    static int configured = -1, sms = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured != dev) {
        e = cudaFuncSetAttribute(k_inner_tc<PH_EULER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(tc::Smem));
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        configured = dev;
    }
    const int ntiles = (P.ncell + tc::TM - 1) / tc::TM;
    const int grid = ntiles < sms ? ntiles : sms;
    k_inner_tc<PH_EULER><<<grid, tc::NT, sizeof(tc::Smem), st>>>(P, X);
    return cudaGetLastError();
}

}  // namespace crkdg
