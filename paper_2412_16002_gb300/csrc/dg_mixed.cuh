// dg_mixed.cuh -- split-precision cRKDG path: FP64 cell averages, FP32 nodal
// deviations, every operator evaluated in FP32.
//
// State of a cell: ubar (FP64, one value per component) and dev (FP32, one per
// node); the polynomial is ubar + (dev - dbar)(x) with dbar the Gauss-weighted
// mean of dev, so the cell average is exactly ubar.
//
// Per stage:
//   * G is evaluated in FP32 (flux, volume term, traces, lift); its deviation part
//     G32 - mean(G32) updates dev, and its average (eq. Gbar, the weighted sum of the
//     FP32 interior-trace fluxes) increments the FP64 stage average of the cell.
//   * The final stage updates ubar with the FP64 sum over the cell's face points of
//     sum_i b_i fhat^(i) (local conservation, Sec. 3.2); each face value is computed
//     identically by both cells, so the global sum is conserved to FP64 round-off.
//   * The scaling limiter keeps FP64 where bounds are decided: the S_K values are
//     screened in FP32 with a rigorous rounding margin, and only cells that the
//     screen cannot clear are evaluated as ubar + (double)(FP32 interpolation) in
//     FP64, where theta is solved and the result verified (the same rounding safety
//     rule as the FP64 path).
#pragma once

#include "dg_core.cuh"

namespace crkdg {

// ----------------------------------------------------------------------------- FP32 physics

template <int PHYS, int DIM>
__device__ __forceinline__ void flux_dir_f(const Params &P, const float *u, int dir, float *f) {
    if constexpr (PHYS == PH_ADV) {
        f[0] = (dir == 0 ? P.f.velx : P.f.vely) * u[0];
    } else if constexpr (PHYS == PH_BURG) {
        f[0] = 0.5f * u[0] * u[0];
    } else if constexpr (DIM == 1) {
        float ri = 1.0f / u[0];
        float w = u[1] * ri;
        float p = P.f.gm1 * (u[2] - 0.5f * u[1] * w);
        f[0] = u[1];
        f[1] = u[1] * w + p;
        f[2] = (u[2] + p) * w;
    } else {
        float ri = 1.0f / u[0];
        float wx = u[1] * ri, wy = u[2] * ri;
        float p = P.f.gm1 * (u[3] - 0.5f * (u[1] * wx + u[2] * wy));
        float wd = dir == 0 ? wx : wy;
        f[0] = u[1 + dir];
        f[1] = u[1] * wd + (dir == 0 ? p : 0.0f);
        f[2] = u[2] * wd + (dir == 1 ? p : 0.0f);
        f[3] = (u[3] + p) * wd;
    }
}

template <int PHYS>
__device__ __forceinline__ void flux_xy_f(const Params &P, const float *u, float *fx, float *fy) {
    if constexpr (PHYS == PH_ADV) {
        fx[0] = P.f.velx * u[0];
        fy[0] = P.f.vely * u[0];
    } else if constexpr (PHYS == PH_BURG) {
        fx[0] = fy[0] = 0.5f * u[0] * u[0];
    } else {
        float ri = 1.0f / u[0];
        float wx = u[1] * ri, wy = u[2] * ri;
        float p = P.f.gm1 * (u[3] - 0.5f * (u[1] * wx + u[2] * wy));
        float ep = u[3] + p;
        fx[0] = u[1];
        fx[1] = u[1] * wx + p;
        fx[2] = u[2] * wx;
        fx[3] = ep * wx;
        fy[0] = u[2];
        fy[1] = u[1] * wy;
        fy[2] = u[2] * wy + p;
        fy[3] = ep * wy;
    }
}

template <int PHYS, int DIM>
__device__ __forceinline__ float speed_dir_f(const Params &P, const float *u, int dir) {
    if constexpr (PHYS == PH_ADV) {
        return fabsf(dir == 0 ? P.f.velx : P.f.vely);
    } else if constexpr (PHYS == PH_BURG) {
        return fabsf(u[0]);
    } else {
        float ri = 1.0f / u[0];
        float kin = DIM == 1 ? u[1] * u[1] : u[1] * u[1] + u[2] * u[2];
        float g = P.f.gamma;
        float p = (g - 1.0f) * (u[DIM + 1] - 0.5f * kin * ri);
        float c2 = g * p * ri;
        float c = c2 > 0.0f ? sqrtf(c2) : 0.0f;
        return fabsf(u[1 + dir] * ri) + c;
    }
}

// Normal flux and the spectral radius |w . nu| + c of one state together (the final stage
// needs both at every face point): one reciprocal and one pressure per state.
template <int PHYS, int DIM>
__device__ __forceinline__ float flux_speed_dir_f(const Params &P, const float *u, int dir, float *f) {
    if constexpr (PHYS != PH_EULER) {
        flux_dir_f<PHYS, DIM>(P, u, dir, f);
        return speed_dir_f<PHYS, DIM>(P, u, dir);
    } else {
        const float ri = 1.0f / u[0];
        float p;
        if constexpr (DIM == 1) {
            const float w = u[1] * ri;
            p = P.f.gm1 * (u[2] - 0.5f * u[1] * w);
            f[0] = u[1];
            f[1] = u[1] * w + p;
            f[2] = (u[2] + p) * w;
        } else {
            const float wx = u[1] * ri, wy = u[2] * ri;
            p = P.f.gm1 * (u[3] - 0.5f * (u[1] * wx + u[2] * wy));
            const float wd = dir == 0 ? wx : wy;
            f[0] = u[1 + dir];
            f[1] = u[1] * wd + (dir == 0 ? p : 0.0f);
            f[2] = u[2] * wd + (dir == 1 ? p : 0.0f);
            f[3] = (u[3] + p) * wd;
        }
        const float c2 = P.f.gamma * p * ri;
        const float c = c2 > 0.0f ? sqrtf(c2) : 0.0f;
        return fabsf(u[1 + dir] * ri) + c;
    }
}

template <int PHYS, int DIM>
__device__ __forceinline__ void boundary_state_f(const Params &P, int side, const float *ui, float *ue) {
    constexpr int M = ncomp(PHYS, DIM);
    int bc = P.bc[side];
    if (bc == BC_DIRICHLET) {
#pragma unroll
        for (int c = 0; c < M; ++c) ue[c] = P.f.bcs[side][c];
    } else {
#pragma unroll
        for (int c = 0; c < M; ++c) ue[c] = ui[c];
        if constexpr (PHYS == PH_EULER) {
            if (bc == BC_REFLECT) ue[1 + side / 2] = -ui[1 + side / 2];
        }
    }
}

// Exterior trace of a boundary face point (FP32): outflow takes the cell average of
// the same stage value, the other conditions as boundary_state_f.
template <int PHYS, int DIM>
__device__ __forceinline__ void exterior_state_f(const Params &P, int side, const float *ui, const float *avg,
                                                 float *ue) {
    constexpr int M = ncomp(PHYS, DIM);
    if (P.bc[side] == BC_OUTFLOW) {
#pragma unroll
        for (int c = 0; c < M; ++c) ue[c] = avg[c];
    } else {
        boundary_state_f<PHYS, DIM>(P, side, ui, ue);
    }
}

// Near vacuum an FP32 density formed as ubar_f + d (ubar_f the FP32 average, d the point's
// deviation) may have lost its sign or most of its digits to rounding; 1 / rho then gives
// an infinite or meaningless velocity.  True when rho is not above 2^-20 (|ubar_f| + |d|),
// beyond which its relative error is below 2^-3: the caller then evaluates that point's
// density (or the whole point) in FP64 from ubar + (double)d.
__device__ __forceinline__ bool rho_ill(float rho, float ubf0, float d0) {
    return !(rho > 9.5367431640625e-07f * (fabsf(ubf0) + fabsf(d0)));
}

// Euler fluxes at a point whose FP32 density is ill-conditioned: the FP64 state ub + (double)d
// (d the FP32 deviations), the FP64 flux, rounded to FP32.  Out of line: it is rare, and the
// kernels that call it are bound by instruction fetch.
template <int DIM>
__device__ __noinline__ void flux_xy_fallback(const Params &P, const double *ub, const float *d, float *fx,
                                                 float *fy) {
    constexpr int M = DIM + 2;
    double u[M], gx[M], gy[M];
#pragma unroll
    for (int c = 0; c < M; ++c) u[c] = ub[c] + (double)d[c];
    if constexpr (DIM == 2) {
        flux_xy<PH_EULER>(P, u, gx, gy);
#pragma unroll
        for (int c = 0; c < M; ++c) {
            fx[c] = (float)gx[c];
            fy[c] = (float)gy[c];
        }
    } else {
        flux_dir<PH_EULER, DIM>(P, u, 0, gx);
#pragma unroll
        for (int c = 0; c < M; ++c) fx[c] = (float)gx[c];
    }
}

// ----------------------------------------------------------------------------- block storage

// Q^3 in 2D (n = 4): node rows are 16-byte aligned float4s, so the line operators read a
// whole row with one shared-memory load; column access goes through transposed copies.
template <class C>
constexpr bool vec4() {
    return C::D == 2 && C::NP == 4;
}

// Largest number of threads of one warp whose shared-memory words share a bank when
// the threads (cell lc, node k < M * parts) read element (k % parts) * ch + q of component
// k / parts's row of their cell, the rows of a component being R words long and the
// components S words apart (word (k / parts) * S + lc * R + (k % parts) * ch + q).  These
// are the per-cell sums over a cell's nodes or face points, one thread per component (or
// per component and chunk); each extra thread on a bank costs one more wavefront.
template <class C>
constexpr int comp_bank_mult(int R, int S, int parts, int ch) {
    int worst = 0;
    for (int w = 0; w < C::NT; w += 32) {
        int cnt[32] = {};
        for (int t = w; t < w + 32 && t < C::NT; ++t) {
            const int lc = t / C::NN, k = t - lc * C::NN;
            if (k >= C::M * parts) continue;
            const int c = k / parts, part = k - c * parts;
            const int b = (c * S + lc * R + part * ch) % 32;
            if (++cnt[b] > worst) worst = cnt[b];
        }
    }
    return worst;
}

// Padding (in words) of the per-component rows of R words of every cell of a block that
// spreads the per-cell sums over the banks: the smallest of 0..31 with the fewest
// wavefronts (with parts > 1 the chunked face sums of the final stage count too).
template <class C>
constexpr int comp_pad(int R, int parts, int ch) {
    int best = 0, bestm = 1 << 30;
    for (int p = 0; p < 32; ++p) {
        const int S = C::NCB * R + p;
        const int m = comp_bank_mult<C>(R, S, 1, 0) + (parts > 1 ? comp_bank_mult<C>(R, S, parts, ch) : 0);
        if (m < bestm) {
            bestm = m;
            best = p;
        }
    }
    return best;
}

// One component's rows (R floats per cell) of a block's cells, followed by PAD unused
// words; S.x[c][lc][q] indexes it like a [NCB][R] array.
template <int NCB, int R, int PAD>
struct PadRows {
    float d[NCB * R + PAD];
    __device__ __forceinline__ float *operator[](int lc) { return d + lc * R; }
    __device__ __forceinline__ const float *operator[](int lc) const { return d + lc * R; }
};

// chunks of the final stage's FP64 face sums per component (see k_final_x)
template <class C>
constexpr int face_parts() {
    return C::NN >= 4 * C::M ? 4 : (C::NN >= 2 * C::M ? 2 : 1);
}

template <class C>
struct alignas(16) SmemX {
    // component-major ([m][cell][...]): a warp's threads (consecutive nodes or face points of
    // consecutive cells) touch consecutive words of one component
    float u[C::M][C::NCB][C::NN];     // node values (or deviations in the limiter)
    float uT[C::M][C::NCB][vec4<C>() ? C::NN : 1];  // the same, transposed (node a*n + b)
    float f[C::D][C::M][C::NCB][C::NN];  // fluxes; with vec4 the y-fluxes are transposed
    // trace fluxes / face corrections; weighted values for the per-cell FP32 means (both
    // padded per component for the per-cell sums)
    PadRows<C::NCB, C::NTR,
            comp_pad<C>(C::NTR, face_parts<C>(), (C::NTR + face_parts<C>() - 1) / face_parts<C>())>
        tf[C::M];
    PadRows<C::NCB, C::NN, comp_pad<C>(C::NN, 1, 0)> w[C::M];
    // the per-cell sums read at most two words per bank (one wavefront, or two where a
    // block's cells cannot all be spread; unpadded they were up to 4-way conflicts)
    static_assert(comp_bank_mult<C>(C::NN, C::NCB * C::NN + comp_pad<C>(C::NN, 1, 0), 1, 0) <= 2,
                  "per-cell sums of the weighted values conflict");
    static_assert(comp_bank_mult<C>(C::NTR,
                                    C::NCB * C::NTR +
                                        comp_pad<C>(C::NTR, face_parts<C>(),
                                                    (C::NTR + face_parts<C>() - 1) / face_parts<C>()),
                                    1, 0) <= 2,
                  "per-cell sums of the face fluxes conflict");
    float ubf[C::NCB][C::M];          // FP32 copy of the averages
    float mean[C::NCB][C::M];
    double gb[C::NCB][C::M];          // FP64 face sums
    double ubd[C::NCB][C::M];         // FP64 averages of the current stage
    float gbf[C::NCB][C::M];          // FP32 average of G (eq. Gbar)
    double kap[C::NTR];               // face-sum weights -sgn * w_pos / h_dir
    float kapf[C::NTR];
    union {  // never live at the same time
        double redd[C::NCB][C::NN][2];
        float al[C::NCB][C::NTR];
        double term[C::M][C::NCB][C::NTR];
    };
    double th[C::NCB][2];
    int fl[C::NCB][C::NN];
    int unsafe[C::NCB];
    int bad[C::NCB];
};

// Gauss weight of node q (normalised: the weights of a cell sum to 1)
template <int DIM, int N>
__device__ __forceinline__ float wnode_f(int q) {
    const NodalTables &T = c_tab[N - 2];
    return DIM == 2 ? T.w2f[q] : T.w1f[q];
}

template <class C>
__device__ __forceinline__ void init_kappa(const Params &P, SmemX<C> &S) {
    const NodalTables &T = c_tab[C::NP - 2];
    for (int fp = threadIdx.x; fp < C::NTR; fp += blockDim.x) {
        int face = fp / C::NF, pos = fp - face * C::NF;
        double wbar = C::D == 2 ? T.w1[pos] : 1.0;
        double rh = face < 2 ? P.rhx : P.rhy;
        S.kap[fp] = ((face & 1) ? -0.5 : 0.5) * wbar * rh;  // -sgn(face) * wbar / h
        S.kapf[fp] = (float)S.kap[fp];
    }
}

// FP32 interpolation of node data q[c][node] of one cell to S_K point p
// q: the cell's node data of component 0; component c starts at q + c * cs.  qT (may be
// null unless n = 4 in 2D): the transposed copy, read as float4 columns.
template <int DIM, int N, int M, int NN>
__device__ __forceinline__ void sk_eval_f(const float *q, const float *qT, int cs, int p, float *v) {
    const NodalTables &T = c_tab[N - 2];
    constexpr int L = nlob(N);
    if constexpr (DIM == 1) {
#pragma unroll
        for (int c = 0; c < M; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int a = 0; a < N; ++a) s = fmaf(T.Iglf[p][a], q[c * cs + a], s);
            v[c] = s;
        }
    } else if (DIM == 2 && N == 4 && p < N * L) {  // row beta as one float4 per component
        int beta = p / L, al = p - beta * L;
#pragma unroll
        for (int c = 0; c < M; ++c) {
            const float4 r = *reinterpret_cast<const float4 *>(q + c * cs + beta * N);
            float s = 0.0f;
            s = fmaf(T.Iglf[al][0], r.x, s);
            s = fmaf(T.Iglf[al][1], r.y, s);
            s = fmaf(T.Iglf[al][2], r.z, s);
            s = fmaf(T.Iglf[al][3], r.w, s);
            v[c] = s;
        }
    } else if (DIM == 2 && N == 4) {  // column beta from the transposed copy
        int rr = p - N * L;
        int beta = rr / L, al = rr - beta * L;
#pragma unroll
        for (int c = 0; c < M; ++c) {
            const float4 r = *reinterpret_cast<const float4 *>(qT + c * cs + beta * N);
            float s = 0.0f;
            s = fmaf(T.Iglf[al][0], r.x, s);
            s = fmaf(T.Iglf[al][1], r.y, s);
            s = fmaf(T.Iglf[al][2], r.z, s);
            s = fmaf(T.Iglf[al][3], r.w, s);
            v[c] = s;
        }
    } else if (p < N * L) {
        int beta = p / L, al = p - beta * L;
#pragma unroll
        for (int c = 0; c < M; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int a = 0; a < N; ++a) s = fmaf(T.Iglf[al][a], q[c * cs + beta * N + a], s);
            v[c] = s;
        }
    } else {
        int r = p - N * L;
        int beta = r / L, al = r - beta * L;
#pragma unroll
        for (int c = 0; c < M; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int b = 0; b < N; ++b) s = fmaf(T.Iglf[al][b], q[c * cs + b * N + beta], s);
            v[c] = s;
        }
    }
}

// ----------------------------------------------------------------------------- G in FP32

// gd: deviation part of G at this node (FP32, cell mean removed); gb: the cell
// average of G as the FP64 sum of the FP32 interior-trace fluxes (eq. Gbar).
template <class C>
__device__ void eval_G_x(const Params &P, SmemX<C> &S, int lc, int node, const float *dv, float *gd,
                         float (&trs)[C::FPT][C::M]) {
    constexpr int DIM = C::D, N = C::NP, PHYS = C::PH;
    constexpr int M = C::M, NN = C::NN, NF = C::NF, NTR = C::NTR, FPT = C::FPT;
    const NodalTables &T = c_tab[N - 2];
    const int a = node % N, b = DIM == 2 ? node / N : 0;
    // S.ubf holds the FP32 copy of the stage averages (written by the caller)
    {
        float u[M], fx[M], fy[M];
#pragma unroll
        for (int c = 0; c < M; ++c) u[c] = S.ubf[lc][c] + dv[c];
        bool ill = false;
        if constexpr (PHYS == PH_EULER) ill = rho_ill(u[0], S.ubf[lc][0], dv[0]);
        if (ill) {  // near vacuum: this node's flux in FP64
            if constexpr (PHYS == PH_EULER) flux_xy_fallback<DIM>(P, S.ubd[lc], dv, fx, fy);
        } else if constexpr (DIM == 2) {
            flux_xy_f<PHYS>(P, u, fx, fy);
        } else {
            flux_dir_f<PHYS, DIM>(P, u, 0, fx);
        }
#pragma unroll
        for (int c = 0; c < M; ++c) {
            S.u[c][lc][node] = u[c];
            S.f[0][c][lc][node] = fx[c];
            if constexpr (vec4<C>()) {
                S.uT[c][lc][a * N + b] = u[c];
                S.f[1][c][lc][a * N + b] = fy[c];  // transposed: column a is contiguous
            } else if constexpr (DIM == 2) {
                S.f[1][c][lc][node] = fy[c];
            }
        }
    }
    __syncthreads();
    float vx[M], vy[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
        if constexpr (vec4<C>()) {
            const float4 fr = *reinterpret_cast<const float4 *>(&S.f[0][c][lc][b * N]);
            const float4 fc = *reinterpret_cast<const float4 *>(&S.f[1][c][lc][a * N]);
            float s = 0.0f, t = 0.0f;
            s = fmaf(T.Dhatf[a][0], fr.x, s);
            s = fmaf(T.Dhatf[a][1], fr.y, s);
            s = fmaf(T.Dhatf[a][2], fr.z, s);
            s = fmaf(T.Dhatf[a][3], fr.w, s);
            t = fmaf(T.Dhatf[b][0], fc.x, t);
            t = fmaf(T.Dhatf[b][1], fc.y, t);
            t = fmaf(T.Dhatf[b][2], fc.z, t);
            t = fmaf(T.Dhatf[b][3], fc.w, t);
            vx[c] = s;
            vy[c] = t;
        } else {
            float s = 0.0f;
#pragma unroll
            for (int q = 0; q < N; ++q) s = fmaf(T.Dhatf[a][q], S.f[0][c][lc][b * N + q], s);
            vx[c] = s;
            if constexpr (DIM == 2) {
                float t = 0.0f;
#pragma unroll
                for (int r = 0; r < N; ++r) t = fmaf(T.Dhatf[b][r], S.f[1][c][lc][r * N + a], t);
                vy[c] = t;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < FPT; ++j) {
        int fp = node + j * NN;
        if (fp < NTR) {
            int face = fp / NF, pos = fp - face * NF;
            const float *l = (face & 1) ? T.lpf : T.lmf;
#pragma unroll
            for (int c = 0; c < M; ++c) {
                float s = 0.0f;
                if constexpr (vec4<C>()) {  // row pos (x faces) or column pos (y faces) as a float4
                    const float4 r = *reinterpret_cast<const float4 *>(face < 2 ? &S.u[c][lc][pos * N]
                                                                                : &S.uT[c][lc][pos * N]);
                    s = fmaf(l[0], r.x, s);
                    s = fmaf(l[1], r.y, s);
                    s = fmaf(l[2], r.z, s);
                    s = fmaf(l[3], r.w, s);
                } else if (DIM == 1 || face < 2) {
#pragma unroll
                    for (int q = 0; q < N; ++q) s = fmaf(l[q], S.u[c][lc][pos * N + q], s);
                } else {
#pragma unroll
                    for (int q = 0; q < N; ++q) s = fmaf(l[q], S.u[c][lc][q * N + pos], s);
                }
                trs[j][c] = s;
            }
            if constexpr (PHYS == PH_EULER) {
                // in a step the stage values are limited and a face point is an S_K point, so
                // its density is >= eps; near vacuum the FP32 interpolation of the node values
                // can lose that to rounding: keep it at least the FP32 value of eps.  (Operator
                // evaluations take unlimited data, whose traces keep their own sign.)
                if (P.mode == MODE_STEP && rho_ill(trs[j][0], S.ubf[lc][0], trs[j][0] - S.ubf[lc][0]))
                    trs[j][0] = fmaxf(trs[j][0], P.scr_eps);
            }
            float f[M];
            flux_dir_f<PHYS, DIM>(P, trs[j], face >> 1, f);
#pragma unroll
            for (int c = 0; c < M; ++c) S.tf[c][lc][fp] = f[c];
        }
    }
    __syncthreads();
    const float rhx = P.f.rhx, rhy = P.f.rhy;
    float g32[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
        float gx = vx[c] - T.liftpf[a] * S.tf[c][lc][NF + b] + T.liftmf[a] * S.tf[c][lc][b];
        float gv = rhx * gx;
        if constexpr (DIM == 2) {
            float gy = vy[c] - T.liftpf[b] * S.tf[c][lc][3 * NF + a] + T.liftmf[b] * S.tf[c][lc][2 * NF + a];
            gv = fmaf(rhy, gy, gv);
        }
        g32[c] = gv;
        S.w[c][lc][node] = wnode_f<DIM, N>(node) * gv;
    }
    __syncthreads();
    for (int c = node; c < M; c += NN) {
        float m = 0.0f, g = 0.0f;
        for (int q = 0; q < NN; ++q) m += S.w[c][lc][q];
        for (int fp = 0; fp < NTR; ++fp) g = fmaf(S.kapf[fp], S.tf[c][lc][fp], g);
        S.mean[lc][c] = m;
        S.gbf[lc][c] = g;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < M; ++c) gd[c] = g32[c] - S.mean[lc][c];
}

// ----------------------------------------------------------------------------- limiter

// FP32 screen of one point: true when the FP32 value v of a point (vb: the FP32
// copy of the cell average) proves that its FP64 evaluation ubar + (double)(v - vbf)
// lies in the bounds.  |FP64 evaluation - v| <= 2^-23 (|v| + |vb|) per component
// (the rounding of ubar to FP32 and of the FP32 sum), doubled here; for Euler it is
// propagated to rho e = E - |m|^2 / (2 rho) to first order, plus 2^-18 (|E| + |m|^2/(2 rho))
// for the FP32 rounding of the formula and the FP64 rounding of the reference test.
template <int PHYS, int DIM>
__device__ __forceinline__ bool screen_ok(const Params &P, const float *v, const float *vb) {
    const float tiny_rel = 2.384185791015625e-07f;  // 2^-22
    const float re_rel = 3.814697265625e-06f;       // 2^-18
    if constexpr (PHYS == PH_EULER) {
        const float epsf = P.f.eps * 1.0000002f;  // >= eps although eps was rounded to FP32
        float dr = tiny_rel * (fabsf(v[0]) + fabsf(vb[0]));
        if (!(v[0] - dr >= epsf) || !(v[0] > 0.0f)) return false;
        float kin = 0.0f, dkin = 0.0f;
#pragma unroll
        for (int d = 1; d <= DIM; ++d) {
            kin += v[d] * v[d];
            dkin += 2.0f * fabsf(v[d]) * tiny_rel * (fabsf(v[d]) + fabsf(vb[d]));
        }
        float de = tiny_rel * (fabsf(v[DIM + 1]) + fabsf(vb[DIM + 1]));
        // correctly rounded reciprocals instead of three quotients: one more rounding of
        // 2^-24 in hk, far inside the 2^-18 allowance below; the error terms are bounds
        // whose own rounding does not matter at this size
        const float inv = __frcp_rn(v[0]), invd = __frcp_rn(v[0] - dr);
        float hk = 0.5f * kin * inv;
        float re = v[DIM + 1] - hk;
        float dre = de + (0.5f * dkin + hk * dr) * invd + re_rel * (fabsf(v[DIM + 1]) + hk);
        return re - dre >= epsf;
    } else {
        float mr = tiny_rel * (fabsf(v[0]) + fabsf(vb[0]));
        return (v[0] - mr >= P.f.lo) && (v[0] + mr <= P.f.hi);
    }
}

// The FP64 evaluation of the represented polynomial at S_K point p:
// ubar + (double)(FP32 interpolation of dev - dbar).  Defines "in the bounds".
template <class C>
__device__ __forceinline__ void eval64_x(SmemX<C> &S, int lc, int p, const double *ub, double *v, float *v32) {
    constexpr int M = C::M;
    float s[M];
    sk_eval_f<C::D, C::NP, M, C::NN>(&S.u[0][lc][0], vec4<C>() ? &S.uT[0][lc][0] : nullptr, C::NCB * C::NN, p, s);
#pragma unroll
    for (int c = 0; c < M; ++c) {
        float d = s[c] - S.mean[lc][c];
        v[c] = ub[c] + (double)d;
        v32[c] = S.ubf[lc][c] + d;
    }
}

// Publishes dev of every node of the block and the FP32 mean of each cell.
template <class C>
__device__ __forceinline__ void publish_dev(const double *ub, const float *dv, SmemX<C> &S, int lc, int node) {
    constexpr int M = C::M, NN = C::NN;
    (void)ub;  // S.ubf already holds the FP32 copy of the averages
#pragma unroll
    for (int c = 0; c < M; ++c) {
        S.u[c][lc][node] = dv[c];
        if constexpr (vec4<C>()) S.uT[c][lc][(node % 4) * 4 + node / 4] = dv[c];
        S.w[c][lc][node] = wnode_f<C::D, C::NP>(node) * dv[c];
    }
    __syncthreads();
    for (int c = node; c < M; c += NN) {
        float m = 0.0f;
        for (int q = 0; q < NN; ++q) m += S.w[c][lc][q];
        S.mean[lc][c] = m;
    }
    __syncthreads();
}

// Scaling limiter of the split representation (block collective).  ub is not
// changed (the limiter keeps averages); dv is rescaled in place.  pts receives
// FP32 values at this thread's S_K points of the limited polynomial.
template <class C>
__device__ void limit_x(const Params &P, const Bufs &B, SmemX<C> &S, int lc, int node, bool active,
                        const double *ub, float *dv, bool check_avg, bool stats, float (&pts)[C::PPT][C::M]) {
    constexpr int DIM = C::D, PHYS = C::PH;
    constexpr int M = C::M, NN = C::NN, NSK = C::NSK, PPT = C::PPT;
    publish_dev(ub, dv, S, lc, node);
    // 1. FP32 screen of the S_K values with a rounding margin
    int unsafe = 0;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        int p = node + j * NN;
        if (p < NSK) {
            float s[M];
            sk_eval_f<DIM, C::NP, M, NN>(&S.u[0][lc][0], vec4<C>() ? &S.uT[0][lc][0] : nullptr, C::NCB * C::NN, p, s);
#pragma unroll
            for (int c = 0; c < M; ++c) {
                float d = s[c] - S.mean[lc][c];
                pts[j][c] = S.ubf[lc][c] + d;
            }
            if (!screen_ok<PHYS, DIM>(P, pts[j], S.ubf[lc])) unsafe = 1;
        }
    }
    S.fl[lc][node] = unsafe;
    __syncthreads();
    if (node == 0) {
        int any = 0;
        for (int q = 0; q < NN; ++q) any |= S.fl[lc][q];
        // the averages' admissibility: the FP32 screen clears it, else the FP64 test decides
        if (check_avg && active && !screen_ok<PHYS, DIM>(P, S.ubf[lc], S.ubf[lc]) && !admissible<PHYS, DIM>(P, ub))
            atomicOr(B.flag, 1);
        S.unsafe[lc] = any;
        S.bad[lc] = 0;
    }
    __syncthreads();
    const bool cell_unsafe = S.unsafe[lc] != 0;
    if (!__syncthreads_or(cell_unsafe)) return;

    // 2. FP64 theta for the cells the screen could not clear
    double th1 = 1.0, th2 = 1.0;
    double pmin = INFINITY, pmax = -INFINITY;
    if (cell_unsafe) {
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            int p = node + j * NN;
            if (p < NSK) {
                double v[M];
                float v32[M];
                eval64_x(S, lc, p, ub, v, v32);
                pmin = (v[0] == v[0]) ? fmin(pmin, v[0]) : -INFINITY;
                pmax = fmax(pmax, v[0]);
            }
        }
    }
    S.redd[lc][node][0] = pmin;
    S.redd[lc][node][1] = pmax;
    __syncthreads();
    if (node == 0 && cell_unsafe) {
        double mn = INFINITY, mx = -INFINITY;
        for (int q = 0; q < NN; ++q) {
            mn = fmin(mn, S.redd[lc][q][0]);
            mx = fmax(mx, S.redd[lc][q][1]);
        }
        double th = 1.0;
        if constexpr (PHYS == PH_EULER) {
            if (mn < P.eps) th = ratio01(ub[0] - P.eps, ub[0] - mn);
        } else {
            if (mx > P.hi) th = fmin(th, ratio01(P.hi - ub[0], mx - ub[0]));
            if (mn < P.lo) th = fmin(th, ratio01(ub[0] - P.lo, ub[0] - mn));
        }
        S.th[lc][0] = th < 1.0 ? th * kMargin : th;
        S.th[lc][1] = 1.0;
    }
    __syncthreads();
    if (cell_unsafe) th1 = S.th[lc][0];
    if constexpr (PHYS == PH_EULER) {
        double pm = INFINITY;
        if (cell_unsafe) {
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                int p = node + j * NN;
                if (p < NSK) {
                    double v[M];
                    float v32[M];
                    eval64_x(S, lc, p, ub, v, v32);
                    if (th1 < 1.0) v[0] = th1 * (v[0] - ub[0]) + ub[0];
                    double re = rho_e<DIM>(v);
                    pm = (re == re) ? fmin(pm, re) : -INFINITY;
                }
            }
        }
        S.redd[lc][node][1] = pm;
        __syncthreads();
        if (node == 0 && cell_unsafe) {
            double mn = INFINITY;
            for (int q = 0; q < NN; ++q) mn = fmin(mn, S.redd[lc][q][1]);
            double reb = rho_e<DIM>(ub);
            S.th[lc][1] = (mn >= P.eps) ? 1.0 : ratio01(reb - P.eps, reb - mn) * kMargin;
        }
        __syncthreads();
        if (cell_unsafe) th2 = S.th[lc][1];
    }
    // 3. rescale the deviations towards the average; verify with the FP64 evaluation
    const bool limited = cell_unsafe && (th1 < 1.0 || th2 < 1.0);
    float dvo[M], dbar[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
        dvo[c] = dv[c];
        dbar[c] = S.mean[lc][c];
    }
    auto apply = [&](double t2) {
        if constexpr (PHYS == PH_EULER) {
            float s0 = (float)(th1 * t2);
            float s1 = (float)t2;
            dv[0] = s0 * (dvo[0] - dbar[0]);
#pragma unroll
            for (int c = 1; c < M; ++c) dv[c] = s1 * (dvo[c] - dbar[c]);
        } else {
            dv[0] = (float)(th1 * t2) * (dvo[0] - dbar[0]);
        }
    };
    double tfin = th2;
    if (limited) apply(th2);
    if (__syncthreads_or(limited)) {
        for (int attempt = 0; attempt <= 4; ++attempt) {
            publish_dev(ub, dv, S, lc, node);
            bool viol = false;
            if (limited) {
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    int p = node + j * NN;
                    if (p < NSK) {
                        double v[M];
                        float v32[M];
                        eval64_x(S, lc, p, ub, v, v32);
#pragma unroll
                        for (int c = 0; c < M; ++c) pts[j][c] = v32[c];
                        if (!point_ok<PHYS, DIM>(P, v)) viol = true;
                    }
                }
            }
            if (viol) S.bad[lc] = 1;
            bool again = __syncthreads_or(viol);
            if (!again || attempt == 4) break;
            bool mine = S.bad[lc] != 0;
            __syncthreads();
            if (node == 0) S.bad[lc] = 0;
            if (mine) {
                tfin = th2 * retry_factor(attempt + 1);
                apply(tfin);
            }
        }
    }
    if (stats && active && node == 0 && limited) {
        double tr = PHYS == PH_EULER ? fmin(th1, tfin) : th1 * tfin;
        atomicAdd(B.nlim, 1ull);
        atomicMin(B.thmin, dbits(tr > 0.0 ? tr : 0.0));
    }
    if constexpr (PHYS == PH_EULER) {
        // cells the screen could not clear are near the bounds: the S_K values handed back
        // (the callers' trial-step rate) are the rounded FP64 evaluation, whose density is
        // >= eps, not the FP32 sum, which near vacuum can be ~0 and make 1 / rho blow up
        if (cell_unsafe) {
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                int p = node + j * NN;
                if (p < NSK) {
                    double v[M];
                    float v32[M];
                    eval64_x(S, lc, p, ub, v, v32);
#pragma unroll
                    for (int c = 0; c < M; ++c) pts[j][c] = (float)v[c];
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------- kernels

template <class C>
__device__ __forceinline__ Bufs scal_of(const MixBufs &X) {
    Bufs B;
    memset(&B, 0, sizeof(B));
    B.un = nullptr;
    B.ustar = nullptr;
    B.unew = nullptr;
    B.tr = nullptr;
    B.flag = X.flag;
    B.nlim = X.nlim;
    B.thmin = X.thmin;
    B.a0 = X.a0;
    B.aux = X.aux;
    B.ord = X.ord;
    return B;
}

template <class C>
__device__ __forceinline__ void load_x(const Params &P, const MixBufs &X, int cell, int node, bool active, double *ub,
                                       float *dv) {
    constexpr int M = C::M;
#pragma unroll
    for (int c = 0; c < M; ++c) {
        if (active) {
            ub[c] = X.ub[(size_t)c * P.ncell + cell];
            dv[c] = X.dv[((size_t)c * P.ncell + cell) * C::NN + node];
        } else {
            ub[c] = (C::PH == PH_EULER && (c == 0 || c == M - 1)) ? 1.0 : (C::PH == PH_EULER ? 0.0 : 0.5 * (P.lo + P.hi));
            dv[c] = 0.0f;
        }
    }
}

// Resident blocks per SM that the inner and final kernels' register budgets are sized
// for.  These kernels are bound by FP32, shared-memory and load latency, not by a pipe,
// so more resident warps pay even at the price of a few spilled registers: 8 blocks of
// 128 threads (Q^3) and 4 of 288 (Q^2) for the inner kernel, 10 and 4 for the final one,
// took the 2048^2 Q^3 step from 19.4 to 15.8 ms and the 1024^2 Q^2 step from 2.75 to
// 2.00 ms (with the padded rows below), against 4 and 2 for both.
template <class C>
constexpr int split_min_blocks() {
    return C::NT > 128 ? 4 : 8;
}
template <class C>
constexpr int split_final_min_blocks() {
    return C::NT > 128 ? 4 : 10;
}

// Inner stages of the split representation (cell-local).
template <class C>
__global__ void __launch_bounds__(C::NT, split_min_blocks<C>()) k_inner_x(Params P, MixBufs X) {
    constexpr int M = C::M, NN = C::NN, NTR = C::NTR, FPT = C::FPT;
    __shared__ SmemX<C> S;
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blockIdx.x * C::NCB + lc;
    const bool active = cell < P.ncell;
    const bool own = active && owned(P, cell);  // counts in the flag, statistics and rate
    const Bufs B = scal_of<C>(X);
    init_kappa<C>(P, S);
    constexpr int CPT = (M + NN - 1) / NN;  // components owned by a component thread
    double ub0[CPT];                         // u^n averages of the owned components (FP64)
    float gbh[MAXS][CPT];                    // averages of G of the owned components (FP32)
    float dv0[M], dvc[M], dacc[M], gd[MAXS][M];
    {
        double ubt[M];
        load_x<C>(P, X, cell, node, active, ubt, dv0);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            int c = node + k * NN;
            ub0[k] = c < M ? ubt[c] : 0.0;
            if (c < M) {
                S.ubd[lc][c] = ub0[k];
                S.ubf[lc][c] = (float)ub0[k];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < M; ++c) dvc[c] = dacc[c] = dv0[c];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXS; ++i) {
        if (i >= P.s) break;
        if (i > 0) {
            // stage averages: FP64 average of u^n plus the FP32 increments (component threads)
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                int c = node + k * NN;
                if (c < M) {
                    float inc = 0.0f;
#pragma unroll
                    for (int j = 0; j < i; ++j)
                        if (P.f.dtA[i][j] != 0.0f) inc = fmaf(P.f.dtA[i][j], gbh[j][k], inc);
                    double v = ub0[k] + (double)inc;
                    S.ubd[lc][c] = v;
                    S.ubf[lc][c] = (float)v;
                }
            }
#pragma unroll
            for (int c = 0; c < M; ++c) {
                float w = dv0[c];
#pragma unroll
                for (int j = 0; j < i; ++j)
                    if (P.f.dtA[i][j] != 0.0f) w = fmaf(P.f.dtA[i][j], gd[j][c], w);
                dvc[c] = w;
            }
            __syncthreads();
            float pts[C::PPT][M];
            limit_x(P, B, S, lc, node, own, S.ubd[lc], dvc, true, true, pts);
        }
        float trs[FPT][M];
        eval_G_x(P, S, lc, node, dvc, gd[i], trs);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            int c = node + k * NN;
            gbh[i][k] = c < M ? S.gbf[lc][c] : 0.0f;
        }
        if (P.mode == MODE_OP_G) {
            if (active)
#pragma unroll
                for (int c = 0; c < M; ++c)
                    X.nod_out[((size_t)c * P.ncell + cell) * NN + node] = (double)S.gbf[lc][c] + (double)gd[i][c];
        } else if (P.f.dtb[i] != 0.0f) {
#pragma unroll
            for (int c = 0; c < M; ++c) dacc[c] = fmaf(P.f.dtb[i], gd[i][c], dacc[c]);
        }
        if (P.slot[i] >= 0 && active) {
            for (int c = node; c < M; c += NN) X.tavg[((size_t)P.slot[i] * M + c) * P.ncell + cell] = S.ubf[lc][c];
            float *dst = X.tr + (size_t)P.slot[i] * M * P.ncell * NTR;
#pragma unroll
            for (int j = 0; j < FPT; ++j) {
                int fp = node + j * NN;
                if (fp < NTR)
#pragma unroll
                    for (int c = 0; c < M; ++c) dst[((size_t)c * P.ncell + cell) * NTR + fp] = trs[j][c];
            }
        }
    }
    if (P.mode != MODE_OP_G && active)
#pragma unroll
        for (int c = 0; c < M; ++c) X.dv_s[((size_t)c * P.ncell + cell) * NN + node] = dacc[c];
}

// Final stage of the split representation: averages from the FP64 sum of
// sum_i b_i fhat^(i) over the face points, deviations from the FP32 lift of
// sum_i b_i (fhat^(i) - f(u_int^(i))); then the limiter and the trial-step rate.
template <class C>
__global__ void __launch_bounds__(C::NT, split_final_min_blocks<C>()) k_final_x(Params P, MixBufs X) {
    constexpr int DIM = C::D, N = C::NP, PHYS = C::PH;
    constexpr int M = C::M, NN = C::NN, NF = C::NF, NTR = C::NTR, FPT = C::FPT;
    __shared__ SmemX<C> S;
    const NodalTables &T = c_tab[N - 2];
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blockIdx.x * C::NCB + lc;
    const bool active = cell < P.ncell;
    const bool own = active && owned(P, cell);  // counts in the flag, statistics and rate
    const int a = node % N, b = DIM == 2 ? node / N : 0;
    // one face point per thread, NF a power of two, whole cells per warp: the NF points of a face
    // are NF consecutive lanes (2D, Q^3)
    constexpr bool kFaceLanes = NTR == NN && (NF & (NF - 1)) == 0 && NF > 1 && 32 % NN == 0;
    const Bufs B = scal_of<C>(X);
    init_kappa<C>(P, S);
    // u^n's averages: thread `node` of a cell updates components node, node + NN, ... (below M)
    constexpr int CT = (M + NN - 1) / NN;
    double ub0[CT];
#pragma unroll
    for (int t = 0; t < CT; ++t) {
        const int c = node + t * NN;
        ub0[t] = (c < M && active) ? X.ub[(size_t)c * P.ncell + cell] : 0.0;
    }
    float dvs[M];  // u^n's deviations plus dt sum_{i<s} b_i G(u^(i)) (written by the inner kernel)
#pragma unroll
    for (int c = 0; c < M; ++c) dvs[c] = active ? X.dv_s[((size_t)c * P.ncell + cell) * NN + node] : 0.0f;
    float dcf[FPT][M], fhs[FPT][M];
#pragma unroll
    for (int j = 0; j < FPT; ++j)
#pragma unroll
        for (int c = 0; c < M; ++c) dcf[j][c] = fhs[j][c] = 0.0f;

    // the trace offsets of this thread's face points and of their partners in the neighbours
    // (-1: a boundary face), the same in every traced stage
    // (element offsets within a component's block, 32-bit: the host keeps ncell * NTR below
    // 2^32 - 1, the marker of a boundary face)
    const size_t cstr = (size_t)P.ncell * NTR;  // component stride of a trace slot
    unsigned toff[FPT], noff[FPT];
#pragma unroll
    for (int j = 0; j < FPT; ++j) {
        const int fp = node + j * NN;
        toff[j] = (unsigned)cell * NTR + fp;
        noff[j] = 0xffffffffu;
        if (fp < NTR && active) {
            const int face = fp / NF, pos = fp - face * NF;
            const int nb = neighbour(P, cell, face);
            if (nb >= 0) noff[j] = (unsigned)nb * NTR + (face ^ 1) * NF + pos;
        }
    }

    for (int i = 0; i < P.s; ++i) {
        if (P.slot[i] < 0) continue;
        const float *tr = X.tr + (size_t)P.slot[i] * M * cstr;
        const float bi = P.f.b[i];
        // per face point: the interior and exterior normal fluxes and the jump u_R - u_L
        float fin[FPT][M], fex[FPT][M], du[FPT][M], sp[FPT];
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            int fp = node + j * NN;
            if (fp < NTR && active) {
                int face = fp / NF;
                float ui[M], ue[M];
#pragma unroll
                for (int c = 0; c < M; ++c) ui[c] = tr[c * cstr + toff[j]];
                if (noff[j] != 0xffffffffu) {
#pragma unroll
                    for (int c = 0; c < M; ++c) ue[c] = tr[c * cstr + noff[j]];
                } else {
                    float av[M];
#pragma unroll
                    for (int c = 0; c < M; ++c) av[c] = X.tavg[((size_t)P.slot[i] * M + c) * P.ncell + cell];
                    exterior_state_f<PHYS, DIM>(P, face, ui, av, ue);
                }
                const bool upper = face & 1;  // the interior state is u_L on an upper face
                const int dir = face >> 1;
#pragma unroll
                for (int c = 0; c < M; ++c) du[j][c] = upper ? ue[c] - ui[c] : ui[c] - ue[c];
                const float si = flux_speed_dir_f<PHYS, DIM>(P, ui, dir, fin[j]);
                const float se = flux_speed_dir_f<PHYS, DIM>(P, ue, dir, fex[j]);
                sp[j] = fmaxf(0.0f, fmaxf(si, se));
            } else {
                sp[j] = 0.0f;
            }
        }
        // alpha of each face: the largest radius over its points
        float alf[FPT];
        if constexpr (kFaceLanes) {  // a face's points sit on NF consecutive lanes: no barrier
#pragma unroll
            for (int j = 0; j < FPT; ++j) {
                alf[j] = sp[j];
#pragma unroll
                for (int o = 1; o < NF; o <<= 1) alf[j] = fmaxf(alf[j], __shfl_xor_sync(0xffffffffu, alf[j], o));
            }
        } else {
#pragma unroll
            for (int j = 0; j < FPT; ++j) {
                const int fp = node + j * NN;
                if (fp < NTR) S.al[lc][fp] = sp[j];
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < FPT; ++j) {
                const int fp = node + j * NN;
                alf[j] = 0.0f;
                if (fp < NTR) {
                    const int face = fp / NF;
#pragma unroll
                    for (int q = 0; q < NF; ++q) alf[j] = fmaxf(alf[j], S.al[lc][face * NF + q]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            int fp = node + j * NN;
            if (fp < NTR && active) {
                const float alpha = alf[j];
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    float fhat = 0.5f * (fin[j][c] + fex[j][c]) - 0.5f * alpha * du[j][c];
                    dcf[j][c] = fmaf(bi, fhat - fin[j][c], dcf[j][c]);
                    fhs[j][c] = fmaf(bi, fhat, fhs[j][c]);
                }
            }
        }
        if constexpr (!kFaceLanes) __syncthreads();  // S.al is rewritten by the next stage
    }
#pragma unroll
    for (int j = 0; j < FPT; ++j) {
        int fp = node + j * NN;
        if (fp < NTR)
#pragma unroll
            for (int c = 0; c < M; ++c) {
                S.tf[c][lc][fp] = dcf[j][c];
            }
    }
    __syncthreads();
    const float rhx = P.f.rhx, rhy = P.f.rhy;
    float corr[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
        float cx = -T.liftpf[a] * S.tf[c][lc][NF + b] + T.liftmf[a] * S.tf[c][lc][b];
        float cv = rhx * cx;
        if constexpr (DIM == 2) {
            float cy = -T.liftpf[b] * S.tf[c][lc][3 * NF + a] + T.liftmf[b] * S.tf[c][lc][2 * NF + a];
            cv = fmaf(rhy, cy, cv);
        }
        corr[c] = cv;
        S.w[c][lc][node] = wnode_f<DIM, N>(node) * cv;
    }
    if (P.mode == MODE_OP_F) {  // F = G + lift(fhat - f_int): nodal FP64 output, no limiter
        if (active)
#pragma unroll
            for (int c = 0; c < M; ++c) {
                size_t k = ((size_t)c * P.ncell + cell) * NN + node;
                X.nod_out[k] = X.nod_in[k] + (double)corr[c];
            }
        return;
    }
    // local conservation (Sec. 3.2): ubar^{n+1} = ubar^n - dt/|K| sum_faces sum_i b_i fhat^(i).
    // The FP32 face sums go to shared memory; one thread per (component, chunk of face
    // points) accumulates its chunk in FP64 (fma with the FP64 weights), and the chunks
    // are added in a fixed order: half the FP64 instructions of one thread per component
    // summing every face point (each costs 64 cycles whatever the active lanes).
    __syncthreads();  // every thread has read the face corrections in S.tf
#pragma unroll
    for (int j = 0; j < FPT; ++j) {
        int fp = node + j * NN;
        if (fp < NTR)
#pragma unroll
            for (int c = 0; c < M; ++c) S.tf[c][lc][fp] = fhs[j][c];
    }
    __syncthreads();
    constexpr int PARTS = face_parts<C>();
    constexpr int CH = (NTR + PARTS - 1) / PARTS;
    for (int k = node; k < M * PARTS; k += NN) {
        const int c = k / PARTS, part = k - c * PARTS;
        double g = 0.0;
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int fp = part * CH + q;
            if (fp < NTR) g = fma(S.kap[fp], (double)S.tf[c][lc][fp], g);
        }
        S.term[c][lc][part] = g;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < CT; ++t) {
        const int c = node + t * NN;
        if (c < M) {
            float m = 0.0f;
            for (int q = 0; q < NN; ++q) m += S.w[c][lc][q];
            S.mean[lc][c] = m;
            double g = S.term[c][lc][0];
#pragma unroll
            for (int part = 1; part < PARTS; ++part) g += S.term[c][lc][part];
            double v = fma(P.dt, g, ub0[t]);
            S.ubd[lc][c] = v;
            S.ubf[lc][c] = (float)v;
        }
    }
    __syncthreads();
    float dvn[M];
    const float fdt = P.f.dt;
#pragma unroll
    for (int c = 0; c < M; ++c) dvn[c] = fmaf(fdt, corr[c] - S.mean[lc][c], dvs[c]);
    if (P.defer_limit) {  // the troubled-cell kernel limits; the averages' admissibility is tested here,
                          // the new averages also go to aux for the indicator
        if (node == 0 && own && !screen_ok<PHYS, DIM>(P, S.ubf[lc], S.ubf[lc]) && !admissible<PHYS, DIM>(P, S.ubd[lc]))
            atomicOr(B.flag, 1);
        if (active) {
            for (int c = node; c < M; c += NN) {
                X.ub_n[(size_t)c * P.ncell + cell] = S.ubd[lc][c];
                X.aux[(size_t)cell * M + c] = S.ubd[lc][c];
            }
#pragma unroll
            for (int c = 0; c < M; ++c) X.dv_n[((size_t)c * P.ncell + cell) * NN + node] = dvn[c];
        }
        return;
    }
    float pts[C::PPT][M];
    limit_x(P, B, S, lc, node, own, S.ubd[lc], dvn, true, true, pts);
    float amax = 0.0f;
#pragma unroll
    for (int j = 0; j < C::PPT; ++j) {
        int p = node + j * NN;
        if (p < C::NSK && own) {
            float r = speed_dir_f<PHYS, DIM>(P, pts[j], 0) * (0.5f * rhx);
            if constexpr (DIM == 2) r = fmaf(speed_dir_f<PHYS, DIM>(P, pts[j], 1), 0.5f * rhy, r);
            amax = fmaxf(amax, r);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    // the rate is FP32-evaluated: widen by 2^-20 before it bounds the FP64 step
    if ((threadIdx.x & 31) == 0 && amax > 0.0f) atomicMax(X.a0, dbits((double)amax * (1.0 + 9.5367431640625e-07)));
    if (active) {
        for (int c = node; c < M; c += NN) X.ub_n[(size_t)c * P.ncell + cell] = S.ubd[lc][c];
#pragma unroll
        for (int c = 0; c < M; ++c) X.dv_n[((size_t)c * P.ncell + cell) * NN + node] = dvn[c];
    }
}

// FP32 screen of the plain indicator's decision for one face-averaged trace deviation
// t, given an FP32 estimate s with |s - t| <= E, the threshold thr and the differences
// of the averages dp, dm (FP32 roundings of FP64 values; sdp, sdm their exact signs).
// The cell keeps t (not troubled) iff |t| <= thr, or t, dp, dm share one sign and
// |t| <= min(|dp|, |dm|).  Every comparison is taken only when it clears the margin
// E + 2^-20 (|x| + |y|), which covers the roundings of thr, dp, dm and of the FP32
// comparisons themselves.  Returns 0 (kept), 1 (troubled) or 2 (undecided).
__device__ __forceinline__ int tvb_screen(float s, float E, float thr, float dp, float dm, int sdp, int sdm) {
    const float as = fabsf(s);
    const float m1 = E + 9.5367431640625e-07f * (as + thr) + 1e-37f;
    if (thr - as > m1) return 0;
    if (!(as - thr > m1)) return 2;
    // |t| > thr >= 0, so t != 0 and has the sign of s
    const int ss = s > 0.0f ? 1 : -1;
    if (sdp != ss || sdm != ss) return 1;
    const float adp = fabsf(dp), adm = fabsf(dm);
    const float m2 = E + 9.5367431640625e-07f * (as + fmaxf(adp, adm)) + 1e-37f;
    if (as - adp > m2 || as - adm > m2) return 1;
    if (adp - as > m2 && adm - as > m2) return 0;
    return 2;
}

// Troubled-cell pass of the split representation, on the unlimited u^{n+1} (X.ub_n,
// X.dv_n, rewritten in place) with its averages in aux.  The decision is the plain
// indicator's (ind_stage 0: taken here; 2: read from tflags; 3: read from tflags and
// combined with the learned probabilities, p > 0.6 troubled, p < 0.4 smooth; 4: taken
// here and combined with the learned probabilities).  Taken here, it is the FP64
// decision on the merged nodal values ubar + (double)(dev - dbar): the face-averaged
// trace deviations are estimated in FP32 from the deviations alone (the average
// cancels in them), with the bound
//   |s - t| <= (n_nodes + 6) 2^-24 sum_q |W_q| |dev_q| + 2^-43 (1 + sum_q |W_q|) (|ubar| + max_q |dev_q|),
// the first term the FP32 weights and dot product, the second the FP64 evaluation
// (merge rounding, dot product, sum of the weights vs 1); a pair the screen cannot
// decide is evaluated in FP64 exactly as on the merged values.  A troubled cell keeps
// its FP64 average and becomes ubar + minmod(c_x, D+x, D-x) xi + minmod(c_y, D+y, D-y) eta,
// its moments c_x, c_y in FP64 from the merged values; the deviations become the FP32
// values of that linear part.  Then the scaling limiter and the trial-step rate.
template <class C>
__global__ void __launch_bounds__(C::NT) k_trouble_x(Params P, MixBufs X) {
    constexpr int DIM = C::D, N = C::NP, PHYS = C::PH, M = C::M, NN = C::NN;
    __shared__ SmemX<C> S;
    __shared__ double sP1[C::NCB][DIM][M];
    __shared__ double sD[C::NCB][DIM][M][2];
    __shared__ int sTr[C::NCB];
    const NodalTables &T = c_tab[N - 2];
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blockIdx.x * C::NCB + lc;
    const bool active = cell < P.ncell;
    const int a = node % N, b = DIM == 2 ? node / N : 0;
    Bufs B = scal_of<C>(X);
    double ub[M];
    float dv[M];
    {
        MixBufs Y = X;
        Y.ub = X.ub_n;
        Y.dv = X.dv_n;
        load_x<C>(P, Y, cell, node, active, ub, dv);
    }
    for (int c = node; c < M; c += NN) {
        S.ubd[lc][c] = ub[c];
        S.ubf[lc][c] = (float)ub[c];
    }
    if (node == 0) sTr[lc] = 0;
    publish_dev(ub, dv, S, lc, node);
    // (direction, component) pairs spread over the cell's threads
    for (int j = node; j < DIM * M && active; j += NN) {
        const int d = j / M, c = j - d * M;
        const double own = S.ubd[lc][c];
        const double lo = nb_average<PHYS, DIM>(P, X.aux, cell, 2 * d, c);
        const double hi = nb_average<PHYS, DIM>(P, X.aux, cell, 2 * d + 1, c);
        const double dp = hi - own, dm = own - lo;
        sD[lc][d][c][0] = dp;
        sD[lc][d][c][1] = dm;
        if (P.ind_stage != 0 && P.ind_stage != 4) continue;
        const float mean = S.mean[lc][c];
        float sR = 0.0f, sL = 0.0f, bR = 0.0f, bL = 0.0f, aR = 0.0f, aL = 0.0f, dmax = 0.0f;
#pragma unroll
        for (int q = 0; q < NN; ++q) {
            const int qa = q % N, qb = DIM == 2 ? q / N : 0;
            const int along = d == 0 ? qa : qb, across = d == 0 ? qb : qa;
            const float wa = DIM == 2 ? T.w1f[across] : 1.0f;
            const float wr = wa * T.lpf[along], wl = wa * T.lmf[along];
            const float e = S.u[c][lc][q] - mean;
            sR = fmaf(wr, e, sR);
            sL = fmaf(wl, e, sL);
            bR = fmaf(fabsf(wr), fabsf(e), bR);
            bL = fmaf(fabsf(wl), fabsf(e), bL);
            aR += fabsf(wr);
            aL += fabsf(wl);
            dmax = fmaxf(dmax, fabsf(e));
        }
        const float base = fabsf(S.ubf[lc][c]) + dmax;
        const float ER = 1.01f * (NN + 6) * 5.9604644775390625e-08f * bR + 1.1368683772161603e-13f * (1.01f + aR) * base;
        const float EL = 1.01f * (NN + 6) * 5.9604644775390625e-08f * bL + 1.1368683772161603e-13f * (1.01f + aL) * base;
        const double thr = P.thr[d];
        const float thrf = P.f.thr[d], dpf = (float)dp, dmf = (float)dm;
        const int sdp = positive_bits(dp) ? 1 : (negative_bits(dp) ? -1 : 0);
        const int sdm = positive_bits(dm) ? 1 : (negative_bits(dm) ? -1 : 0);
        // the left deviation is ubar - avg_face(u_L) = -(face-averaged dev)
        const int rR = tvb_screen(sR, ER, thrf, dpf, dmf, sdp, sdm);
        const int rL = tvb_screen(-sL, EL, thrf, dpf, dmf, sdp, sdm);
        int trouble = (rR == 1 || rL == 1) ? 1 : 0;
        if (!trouble && (rR == 2 || rL == 2)) {  // FP64 on the merged values
            double fr = 0.0, fl = 0.0;
            for (int q = 0; q < NN; ++q) {
                const double v = own + (double)(S.u[c][lc][q] - mean);
                if constexpr (DIM == 2) {
                    fr = fma(T.trw2[d][0][q], v, fr);
                    fl = fma(T.trw2[d][1][q], v, fl);
                } else {
                    fr = fma(T.lp[q], v, fr);
                    fl = fma(T.lm[q], v, fl);
                }
            }
            const double utR = fr - own, utL = own - fl;
            const bool thr_ok = thr >= 0.0;
            trouble = (tvb_changes(utR, dp, dm, thr, thr_ok) || tvb_changes(utL, dp, dm, thr, thr_ok)) ? 1 : 0;
        }
        if (trouble) atomicOr(&sTr[lc], 1);
    }
    __syncthreads();
    bool troubled = active && ((P.ind_stage == 0 || P.ind_stage == 4) ? sTr[lc] != 0 : X.tflags[cell] != 0);
    if ((P.ind_stage == 3 || P.ind_stage == 4) && active) {
        const float pr = X.prob[cell];
        troubled = pr > 0.6f ? true : (pr < 0.4f ? false : troubled);
    }
    if (node == 0 && active) {
        if (P.ind_stage != 2) X.tflags[cell] = troubled ? 1 : 0;
        if (troubled) atomicAdd(X.ntrb, 1ull);
    }
    if (troubled) {  // the same value for all threads of the cell
        for (int j = node; j < DIM * M; j += NN) {
            const int d = j / M, c = j - d * M;
            const double own = S.ubd[lc][c];
            const float mean = S.mean[lc][c];
            double p1 = 0.0;
            for (int q = 0; q < NN; ++q) {
                const double v = own + (double)(S.u[c][lc][q] - mean);
                p1 = fma(DIM == 2 ? T.pm2[d][q] : T.pm1[q], v, p1);
            }
            sP1[lc][d][c] = minmod3_bits(p1, sD[lc][d][c][0], sD[lc][d][c][1]);
        }
    }
    __syncthreads();
    if (troubled) {
#pragma unroll
        for (int c = 0; c < M; ++c) {
            double v = sP1[lc][0][c] * T.xg[a];
            if constexpr (DIM == 2) v = fma(sP1[lc][1][c], T.xg[b], v);
            dv[c] = (float)v;
        }
    }
    float pts[C::PPT][M];
    limit_x(P, B, S, lc, node, active, S.ubd[lc], dv, false, true, pts);
    const float rhx = P.f.rhx, rhy = P.f.rhy;
    float amax = 0.0f;
#pragma unroll
    for (int j = 0; j < C::PPT; ++j) {
        int p = node + j * NN;
        if (p < C::NSK && active) {
            float r = speed_dir_f<PHYS, DIM>(P, pts[j], 0) * (0.5f * rhx);
            if constexpr (DIM == 2) r = fmaf(speed_dir_f<PHYS, DIM>(P, pts[j], 1), 0.5f * rhy, r);
            amax = fmaxf(amax, r);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && amax > 0.0f) atomicMax(X.a0, dbits((double)amax * (1.0 + 9.5367431640625e-07)));
    if (active)
#pragma unroll
        for (int c = 0; c < M; ++c) X.dv_n[((size_t)c * P.ncell + cell) * NN + node] = dv[c];
}

// FP64 nodal -> (ubar, dev), then (optionally) the limiter.
template <class C>
__global__ void __launch_bounds__(C::NT) k_split_x(Params P, MixBufs X) {
    constexpr int DIM = C::D, N = C::NP, M = C::M, NN = C::NN;
    const NodalTables &T = c_tab[N - 2];
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blockIdx.x * C::NCB + lc;
    const bool active = cell < P.ncell;
    double u[M];
    __shared__ double su[C::NCB][M][NN];
    __shared__ double sub[C::NCB][M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
        u[c] = active ? X.nod_in[((size_t)c * P.ncell + cell) * NN + node] : 1.0;
        su[lc][c][node] = u[c];
    }
    __syncthreads();
    for (int c = node; c < M; c += NN) {
        double s = 0.0;
        for (int q = 0; q < NN; ++q) s = fma(DIM == 2 ? T.w2[q] : T.w1[q], su[lc][c][q], s);
        sub[lc][c] = s;
    }
    __syncthreads();
    if (active) {
        for (int c = node; c < M; c += NN) X.ub_n[(size_t)c * P.ncell + cell] = sub[lc][c];
#pragma unroll
        for (int c = 0; c < M; ++c)
            X.dv_n[((size_t)c * P.ncell + cell) * NN + node] = (float)(u[c] - sub[lc][c]);
    }
}

// Trial-step rate at S_K point p of the published split state (deviations and their mean in
// S.u / S.mean, FP32 averages in S.ubf, FP64 averages ub): sum_d radius_d / (2 h_d) of the
// FP32 value, and near vacuum of the FP64 evaluation rounded to FP32.
template <class C>
__device__ __forceinline__ float rate_point_x(const Params &P, SmemX<C> &S, int lc, int p, const double *ub) {
    constexpr int DIM = C::D, PHYS = C::PH, M = C::M;
    float s[M], v32[M];
    sk_eval_f<C::D, C::NP, M, C::NN>(&S.u[0][lc][0], vec4<C>() ? &S.uT[0][lc][0] : nullptr, C::NCB * C::NN, p, s);
#pragma unroll
    for (int c = 0; c < M; ++c) v32[c] = S.ubf[lc][c] + (s[c] - S.mean[lc][c]);
    if constexpr (PHYS == PH_EULER) {
        if (rho_ill(v32[0], S.ubf[lc][0], v32[0] - S.ubf[lc][0])) {
            double v[M];
            eval64_x(S, lc, p, ub, v, v32);
#pragma unroll
            for (int c = 0; c < M; ++c) v32[c] = (float)v[c];
        }
    }
    float r = speed_dir_f<PHYS, DIM>(P, v32, 0) * (0.5f * P.f.rhx);
    if constexpr (DIM == 2) r = fmaf(speed_dir_f<PHYS, DIM>(P, v32, 1), 0.5f * P.f.rhy, r);
    return r;
}

// The largest rate of a block's warps into X.a0, widened by 2^-20 (the rate is FP32-evaluated)
// before it bounds the FP64 step.
__device__ __forceinline__ void post_rate_x(const MixBufs &X, float amax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && amax > 0.0f) atomicMax(X.a0, dbits((double)amax * (1.0 + 9.5367431640625e-07)));
}

// (ubar, dev) -> FP64 nodal values ubar + (dev - dbar).
template <class C>
__global__ void __launch_bounds__(C::NT) k_merge_x(Params P, MixBufs X) {
    constexpr int M = C::M, NN = C::NN;
    __shared__ SmemX<C> S;
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blockIdx.x * C::NCB + lc;
    const bool active = cell < P.ncell;
    double ub[M];
    float dv[M];
    load_x<C>(P, X, cell, node, active, ub, dv);
    for (int c = node; c < M; c += NN) S.ubf[lc][c] = (float)ub[c];
    publish_dev(ub, dv, S, lc, node);
    if (active)
#pragma unroll
        for (int c = 0; c < M; ++c)
            X.nod_out[((size_t)c * P.ncell + cell) * NN + node] = ub[c] + (double)(dv[c] - S.mean[lc][c]);
}

// Limiter of (ubar, dev) in place (after set-up).
template <class C>
__global__ void __launch_bounds__(C::NT) k_limit_x(Params P, MixBufs X) {
    constexpr int M = C::M, NN = C::NN;
    __shared__ SmemX<C> S;
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blockIdx.x * C::NCB + lc;
    const bool active = cell < P.ncell;
    const bool own = active && owned(P, cell);  // counts in the flag, statistics and rate
    const Bufs B = scal_of<C>(X);
    double ub[M];
    float dv[M], pts[C::PPT][M];
    load_x<C>(P, X, cell, node, active, ub, dv);
    for (int c = node; c < M; c += NN) {
        S.ubd[lc][c] = ub[c];
        S.ubf[lc][c] = (float)ub[c];
    }
    __syncthreads();
    limit_x(P, B, S, lc, node, own, S.ubd[lc], dv, false, false, pts);
    if (P.mode == MODE_RATE) {  // the trial-step rate of the limited state (k_scan_x's rate pass):
                                // the limiter left the final deviations published
        float amax = 0.0f;
#pragma unroll
        for (int j = 0; j < C::PPT; ++j) {
            const int p = node + j * NN;
            if (p < C::NSK && own) amax = fmaxf(amax, rate_point_x<C>(P, S, lc, p, S.ubd[lc]));
        }
        post_rate_x(X, amax);
    }
    if (active)
#pragma unroll
        for (int c = 0; c < M; ++c) X.dv_n[((size_t)c * P.ncell + cell) * NN + node] = dv[c];
}

// Trial-step rate (FP32 S_K values, widened) and bound margins (FP64 evaluation).
template <class C>
__global__ void __launch_bounds__(C::NT) k_scan_x(Params P, MixBufs X) {
    constexpr int DIM = C::D, PHYS = C::PH, M = C::M, NN = C::NN;
    __shared__ SmemX<C> S;
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blockIdx.x * C::NCB + lc;
    const bool active = cell < P.ncell;
    const bool own = active && owned(P, cell);  // counts in the flag, statistics and rate
    double ub[M];
    float dv[M];
    load_x<C>(P, X, cell, node, active, ub, dv);
    for (int c = node; c < M; c += NN) S.ubf[lc][c] = (float)ub[c];
    publish_dev(ub, dv, S, lc, node);
    float amax = 0.0f;
    double m0 = INFINITY, m1 = INFINITY;
    const float rhx = P.f.rhx, rhy = P.f.rhy;
    const bool margins = P.mode != MODE_RATE;
#pragma unroll
    for (int j = 0; j < C::PPT; ++j) {
        int p = node + j * NN;
        if (p < C::NSK && own) {
            if (!margins) {
                amax = fmaxf(amax, rate_point_x<C>(P, S, lc, p, ub));
                continue;
            }
            double v[M];
            float v32[M];
            eval64_x(S, lc, p, ub, v, v32);
            if constexpr (PHYS == PH_EULER) {
                if (rho_ill(v32[0], S.ubf[lc][0], v32[0] - S.ubf[lc][0])) {  // near vacuum: FP64
#pragma unroll
                    for (int c = 0; c < M; ++c) v32[c] = (float)v[c];
                }
            }
            float r = speed_dir_f<PHYS, DIM>(P, v32, 0) * (0.5f * rhx);
            if constexpr (DIM == 2) r = fmaf(speed_dir_f<PHYS, DIM>(P, v32, 1), 0.5f * rhy, r);
            amax = fmaxf(amax, r);
            double a0m, a1m;
            if constexpr (PHYS == PH_EULER) {
                a0m = v[0] - P.eps;
                a1m = rho_e<DIM>(v) - P.eps;
            } else {
                a0m = v[0] - P.lo;
                a1m = P.hi - v[0];
            }
            m0 = (a0m == a0m) ? fmin(m0, a0m) : -INFINITY;
            m1 = (a1m == a1m) ? fmin(m1, a1m) : -INFINITY;
        }
    }
    unsigned long long k0 = ordbits(m0), k1 = ordbits(m1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        if (margins) {
            k0 = umin64(k0, __shfl_xor_sync(0xffffffffu, k0, o));
            k1 = umin64(k1, __shfl_xor_sync(0xffffffffu, k1, o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        if (amax > 0.0f) atomicMax(X.a0, dbits((double)amax * (1.0 + 9.5367431640625e-07)));
        if (margins) {
            atomicMin(&X.ord[0], k0);
            atomicMin(&X.ord[1], k1);
        }
    }
}

// Features of the learned indicator from the split state of the unlimited u^{n+1}
// (2D Euler; one thread per cell): the stencil part from the FP64 averages in aux, as
// the FP64 feature kernel; the first moments c_10, c_01 from the FP32 deviations,
// sum_q ((3 w_a) w_b) x_a (dev_q - dbar) (the average's contribution is zero), in FP32.
// The plain decision is left to the troubled-cell pass (ind_stage 4).
template <class C>
__global__ void __launch_bounds__(128) k_features_x(Params P, MixBufs X) {
    constexpr int DIM = C::D, N = C::NP, PHYS = C::PH, M = C::M, NN = C::NN;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (DIM != 2 || PHYS != PH_EULER) {
        return;
    } else {
        if (cell >= P.ncell) return;
        const NodalTables &T = c_tab[N - 2];
        double v[9][M], scale[M];
        float *f = X.feat + (size_t)cell * 44;
        stencil_features<PHYS>(P, X.aux, cell, f, v, scale);
#pragma unroll
        for (int c = 0; c < M; ++c) {
            const float *dv = X.dv_n + ((size_t)c * P.ncell + cell) * NN;
            float d[NN];
#pragma unroll
            for (int q = 0; q < NN; ++q) d[q] = dv[q];
            float dbar = 0.0f;
#pragma unroll
            for (int q = 0; q < NN; ++q) dbar = fmaf(T.w2f[q], d[q], dbar);
            float cx = 0.0f, cy = 0.0f;
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                const float e = d[q] - dbar;
                cx = fmaf(T.momxf[q], e, cx);
                cy = fmaf(T.momyf[q], e, cy);
            }
            const float sc = (float)scale[c];
            f[36 + 2 * c] = cx * sc;
            f[37 + 2 * c] = cy * sc;
        }
    }
}

// Cell averages: aux[cell][m] = ubar
template <class C>
__global__ void k_avg_x(Params P, MixBufs X) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.ncell * C::M) return;
    int cell = t / C::M, c = t - cell * C::M;
    X.aux[t] = X.ub[(size_t)c * P.ncell + cell];
}

template <int DIM, int N, int PHYS>
cudaError_t launch_one_x(int kernel, int nblocks, cudaStream_t st, const Params &P, const MixBufs &X) {
    using C = Cfg<DIM, N, PHYS>;
    switch (kernel) {
    case KX_SPLIT: k_split_x<C><<<nblocks, C::NT, 0, st>>>(P, X); break;
    case KX_MERGE: k_merge_x<C><<<nblocks, C::NT, 0, st>>>(P, X); break;
    case KX_LIMIT: k_limit_x<C><<<nblocks, C::NT, 0, st>>>(P, X); break;
    case KX_INNER: k_inner_x<C><<<nblocks, C::NT, 0, st>>>(P, X); break;
    case KX_FINAL: k_final_x<C><<<nblocks, C::NT, 0, st>>>(P, X); break;
    case KX_SCAN: k_scan_x<C><<<nblocks, C::NT, 0, st>>>(P, X); break;
    case KX_TROUBLE: k_trouble_x<C><<<nblocks, C::NT, 0, st>>>(P, X); break;
    case KX_FEATURES: k_features_x<C><<<(P.ncell + 127) / 128, 128, 0, st>>>(P, X); break;
    case KX_AVG: {
        int tot = P.ncell * C::M;
        k_avg_x<C><<<(tot + 255) / 256, 256, 0, st>>>(P, X);
        break;
    }
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int DIM>
cudaError_t launch_dim_x(int kernel, int n, int phys, int nblocks, cudaStream_t st, const Params &P,
                         const MixBufs &X) {
#define CRKDG_CASE_X(NV, PV) \
    if (n == NV && phys == PV) return launch_one_x<DIM, NV, PV>(kernel, nblocks, st, P, X);
    CRKDG_CASE_X(2, PH_ADV) CRKDG_CASE_X(2, PH_BURG) CRKDG_CASE_X(2, PH_EULER)
    CRKDG_CASE_X(3, PH_ADV) CRKDG_CASE_X(3, PH_BURG) CRKDG_CASE_X(3, PH_EULER)
    CRKDG_CASE_X(4, PH_ADV) CRKDG_CASE_X(4, PH_BURG) CRKDG_CASE_X(4, PH_EULER)
#undef CRKDG_CASE_X
    return cudaErrorInvalidValue;
}

}  // namespace crkdg
