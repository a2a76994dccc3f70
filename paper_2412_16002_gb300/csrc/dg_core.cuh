// dg_core.cuh -- device code of the FP64 cRKDG path (arXiv 2412.16002).
//
// Included by exactly one translation unit per dimension (dg_1d.cu, dg_2d.cu),
// each of which owns its copy of the constant tables.
//
// Work decomposition: one thread per (cell, node).  A block holds NCB cells of
// n^d nodes each; the line operators (volume term, traces, lift, S_K
// interpolation) exchange node data through shared memory.  Per-cell
// reductions (average, min/max over S_K) are taken by one leader thread per
// cell in a fixed order, so every result is deterministic.
//
// Nodal Q^k form of the operators (collocation at the Gauss points, exact
// diagonal mass matrix), per x-line of a cell with traces u_L = sum_a l_a(-1) u_a,
// u_R = sum_a l_a(+1) u_a:
//   G_a = (2/h) [ sum_q Dhat[a][q] f_q - l_a(+1)/w_a f(u_R) + l_a(-1)/w_a f(u_L) ]
// (Sec. 2.1 with the (k+1)-point Gauss rule); in 2D the y-lines add the same
// term.  F replaces f(u_R), f(u_L) by the Lax--Friedrichs flux (eq. dxDG), so
// F = G + lift(fhat - f(u_int)); the final kernel adds exactly that correction.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dg_types.h"

namespace crkdg {

static __constant__ NodalTables c_tab[3];  // n = 2, 3, 4

// ----------------------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long u) { return __longlong_as_double((long long)u); }
// order-preserving map of a double onto uint64 (for atomicMin over signed values)
__device__ __forceinline__ unsigned long long ordbits(double x) {
    unsigned long long u = dbits(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// Comparisons and min/max that need no FP64 arithmetic run on the integer units: the
// FP64 pipe of this part takes one warp instruction per 64 cycles whatever the number
// of active lanes, while a 64-bit integer compare-and-select costs a few ALU issues.
// Keys of +inf and -inf under ordbits.
constexpr unsigned long long kKeyPosInf = 0xfff0000000000000ull;
constexpr unsigned long long kKeyNegInf = 0x000fffffffffffffull;
// inverse of ordbits
__device__ __forceinline__ double ordbits_inv(unsigned long long k) {
    return bitsd((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k);
}
// x != 0.0 on the integer units (NaN counts as non-zero, as for the comparison)
__device__ __forceinline__ bool nonzero_bits(double x) { return (dbits(x) << 1) != 0ull; }
__device__ __forceinline__ bool isnan_bits(double x) {
    return (dbits(x) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
}
__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
// x > 0.0 (false for NaN)
__device__ __forceinline__ bool positive_bits(double x) {
    long long b = (long long)dbits(x);
    return b > 0ll && b <= 0x7ff0000000000000ll;
}
// x >= y for y > 0 (false when x is NaN)
__device__ __forceinline__ bool ge_pos_bits(double x, double y) {
    long long b = (long long)dbits(x);
    return b >= (long long)dbits(y) && b <= 0x7ff0000000000000ll;
}
// t < 1.0 for t in [0, 1] (a limiter's scaling factor)
__device__ __forceinline__ bool below_one(double t) { return (dbits(t) & 0x7fffffffffffffffull) < 0x3ff0000000000000ull; }
// fmax of two non-negative doubles (a NaN operand is ignored, as by fmax)
__device__ __forceinline__ double fmax_nonneg(double a, double b) {
    if (isnan_bits(a)) return b;
    if (isnan_bits(b)) return a;
    return bitsd(umax64(dbits(a), dbits(b)));
}

// 1/x by the Newton-Raphson iteration r <- r + r (1 - x r) (quadratic convergence) from
// the hardware's approximate reciprocal (rcp.approx.ftz.f64); two steps reach double
// precision (within an ulp of the rounded quotient).  Arguments outside [2^-1000,
// 2^1001) in magnitude (zero, subnormal, huge, inf, NaN) take the IEEE division.  On this
// part a dependent FP64 operation costs 64 cycles and the IEEE reciprocal about seven.
__device__ __forceinline__ double recip_nr(double x) {
    const unsigned e = (unsigned)(dbits(x) >> 52) & 0x7ffu;
    if (e < 1023u - 1000u || e > 1023u + 1000u) return 1.0 / x;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double t = fma(-x, r, 1.0);
    r = fma(r, t, r);
    t = fma(-x, r, 1.0);
    return fma(r, t, r);
}

// theta = num/den clamped to [0, 1]; a non-positive denominator gives 0
__device__ __forceinline__ double ratio01(double num, double den) {
    if (!(den > 0.0)) return 0.0;
    double t = num * recip_nr(den);
    if (!(t >= 0.0)) t = 0.0;
    return t > 1.0 ? 1.0 : t;
}

// ----------------------------------------------------------------------------- physics


// Euler flux . e_dir and spectral radius given ri = 1/rho, written with explicit
// roundings (fma, __dmul_rn, __dadd_rn): the compiler cannot contract them
// differently where they are inlined, so a trace's flux stored by the inner kernel
// equals, bit for bit, the same flux recomputed by the final kernel.
template <int DIM>
__device__ __forceinline__ void euler_flux_ri(const Params &P, const double *u, int dir, double ri, double *f) {
    const double gm1 = P.gamma - 1.0;
    if constexpr (DIM == 1) {
        double w = __dmul_rn(u[1], ri);
        double p = __dmul_rn(gm1, fma(-0.5 * u[1], w, u[2]));
        f[0] = u[1];
        f[1] = fma(u[1], w, p);
        f[2] = __dmul_rn(__dadd_rn(u[2], p), w);
    } else {
        double wx = __dmul_rn(u[1], ri), wy = __dmul_rn(u[2], ri);
        double p = __dmul_rn(gm1, fma(-0.5, fma(u[1], wx, __dmul_rn(u[2], wy)), u[3]));
        double wd = dir == 0 ? wx : wy;
        f[0] = u[1 + dir];
        f[1] = dir == 0 ? fma(u[1], wd, p) : __dmul_rn(u[1], wd);
        f[2] = dir == 1 ? fma(u[2], wd, p) : __dmul_rn(u[2], wd);
        f[3] = __dmul_rn(__dadd_rn(u[3], p), wd);
    }
}
template <int DIM>
__device__ __forceinline__ double euler_speed_ri(const Params &P, const double *u, int dir, double ri) {
    double kin = DIM == 1 ? __dmul_rn(u[1], u[1]) : fma(u[1], u[1], __dmul_rn(u[2], u[2]));
    double p = __dmul_rn(P.gamma - 1.0, fma(-0.5 * kin, ri, u[DIM + 1]));
    double c2 = __dmul_rn(__dmul_rn(P.gamma, p), ri);
    double c = positive_bits(c2) ? sqrt(c2) : 0.0;
    return __dadd_rn(fabs(__dmul_rn(u[1 + dir], ri)), c);
}

// flux f(u) . e_dir  (eq. claws; Euler eq. Euler, Euler-2)
template <int PHYS, int DIM>
__device__ __forceinline__ void flux_dir(const Params &P, const double *u, int dir, double *f) {
    if constexpr (PHYS == PH_ADV) {
        f[0] = (dir == 0 ? P.velx : P.vely) * u[0];
    } else if constexpr (PHYS == PH_BURG) {
        f[0] = 0.5 * u[0] * u[0];
    } else {
        euler_flux_ri<DIM>(P, u, dir, recip_nr(u[0]), f);
    }
}

// both directions with one reciprocal (2D)
template <int PHYS>
__device__ __forceinline__ void flux_xy(const Params &P, const double *u, double *fx, double *fy) {
    if constexpr (PHYS == PH_ADV) {
        fx[0] = P.velx * u[0];
        fy[0] = P.vely * u[0];
    } else if constexpr (PHYS == PH_BURG) {
        fx[0] = fy[0] = 0.5 * u[0] * u[0];
    } else {
        double ri = recip_nr(u[0]);
        double wx = u[1] * ri, wy = u[2] * ri;
        double p = (P.gamma - 1.0) * (u[3] - 0.5 * (u[1] * wx + u[2] * wy));
        double ep = u[3] + p;
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

// spectral radius of df/du . e_dir (alpha of the LF flux, a0 of Sec. 2.1)
template <int PHYS, int DIM>
__device__ __forceinline__ double speed_dir(const Params &P, const double *u, int dir) {
    if constexpr (PHYS == PH_ADV) {
        return fabs(dir == 0 ? P.velx : P.vely);
    } else if constexpr (PHYS == PH_BURG) {
        return fabs(u[0]);
    } else {
        return euler_speed_ri<DIM>(P, u, dir, recip_nr(u[0]));
    }
}

// flux_dir and speed_dir given the reciprocal ri = 1/rho of the state (Euler; other
// fluxes ignore it): the same values as flux_dir and speed_dir, one division fewer
// when a state needs both.
template <int PHYS, int DIM>
__device__ __forceinline__ void flux_dir_ri(const Params &P, const double *u, int dir, double ri, double *f) {
    if constexpr (PHYS != PH_EULER) {
        flux_dir<PHYS, DIM>(P, u, dir, f);
    } else {
        euler_flux_ri<DIM>(P, u, dir, ri, f);
    }
}
template <int PHYS, int DIM>
__device__ __forceinline__ double speed_dir_ri(const Params &P, const double *u, int dir, double ri) {
    if constexpr (PHYS != PH_EULER) {
        return speed_dir<PHYS, DIM>(P, u, dir);
    } else {
        return euler_speed_ri<DIM>(P, u, dir, ri);
    }
}
template <int PHYS>
__device__ __forceinline__ double recip_rho(const double *u) {
    if constexpr (PHYS == PH_EULER) return recip_nr(u[0]);
    return 0.0;
}
// both for one state; returns the spectral radius
template <int PHYS, int DIM>
__device__ __forceinline__ double flux_speed_dir(const Params &P, const double *u, int dir, double *f) {
    double ri = recip_rho<PHYS>(u);
    flux_dir_ri<PHYS, DIM>(P, u, dir, ri, f);
    return speed_dir_ri<PHYS, DIM>(P, u, dir, ri);
}

// Trial-step rate at one point: sum over directions of lambda_d / h_d, so that
// dt = CFL / max rate (eq. numerical_experiment:CFL, directional radii summed in 2D).
// The Euler form shares the reciprocal and the sound speed between the directions
// (the same values as speed_dir per direction).
template <int PHYS, int DIM>
__device__ __forceinline__ double sk_rate(const Params &P, const double *u) {
    if constexpr (PHYS == PH_EULER) {
        double ri = recip_nr(u[0]);
        double kin = DIM == 1 ? u[1] * u[1] : u[1] * u[1] + u[2] * u[2];
        double p = (P.gamma - 1.0) * (u[DIM + 1] - 0.5 * kin * ri);
        double c2 = P.gamma * p * ri;
        double c = positive_bits(c2) ? sqrt(c2) : 0.0;
        double r = (fabs(u[1] * ri) + c) * (0.5 * P.rhx);
        if constexpr (DIM == 2) r = fma(fabs(u[2] * ri) + c, 0.5 * P.rhy, r);
        return r;
    } else {
        double r = speed_dir<PHYS, DIM>(P, u, 0) * (0.5 * P.rhx);
        if constexpr (DIM == 2) r = fma(speed_dir<PHYS, DIM>(P, u, 1), 0.5 * P.rhy, r);
        return r;
    }
}

// rho e = E - |m|^2 / (2 rho)   (eq. Euler-limiter2)
template <int DIM>
__device__ __forceinline__ double rho_e(const double *u) {
    double kin = DIM == 1 ? u[1] * u[1] : u[1] * u[1] + u[2] * u[2];
    return u[DIM + 1] - (0.5 * kin) * recip_nr(u[0]);
}

// The exact theta_2 of one S_K point (the alternative to eq. Euler-limiter2's concavity ratio):
// along u(t) = ub + t (u - ub) the density, momentum and energy are linear in t, so with
// rho(t) > 0, rho e(u(t)) >= eps <=> h(t) = (E(t) - eps) rho(t) - |m(t)|^2 / 2 >= 0, a quadratic
// a t^2 + b t + c.  h(0) = rho_bar (rho e(ub) - eps) > 0 for an admissible average and h(1) < 0
// at a violating point: one root in (0, 1), taken in the cancellation-free form
// q = -(b + sign(b) sqrt(b^2 - 4ac)) / 2, roots q / a and c / q.  1 when h(1) >= 0, 0 when the
// average is not strictly inside.  FP64, IEEE division and square root (rare: limited cells).
template <int DIM>
__device__ double theta2_point(const double *ub, const double *u, double eps) {
    const double dr = u[0] - ub[0], dE = u[DIM + 1] - ub[DIM + 1];
    double mm = 0.0, md = 0.0, dd = 0.0;
#pragma unroll
    for (int d = 1; d <= DIM; ++d) {
        const double dm = u[d] - ub[d];
        mm += ub[d] * ub[d];
        md += ub[d] * dm;
        dd += dm * dm;
    }
    const double c = (ub[DIM + 1] - eps) * ub[0] - 0.5 * mm;
    const double b = (ub[DIM + 1] - eps) * dr + dE * ub[0] - md;
    const double a = dE * dr - 0.5 * dd;
    if (!(c > 0.0)) return 0.0;
    if (a + b + c >= 0.0) return 1.0;
    double disc = b * b - 4.0 * a * c;
    if (disc < 0.0) disc = 0.0;
    const double q = -0.5 * (b + (b >= 0.0 ? sqrt(disc) : -sqrt(disc)));
    double best = 2.0;
    if (a != 0.0) {
        const double r = q / a;
        if (r > 0.0 && r < 1.0 && r < best) best = r;
    }
    if (q != 0.0) {
        const double r = c / q;
        if (r > 0.0 && r < 1.0 && r < best) best = r;
    }
    return best <= 1.0 ? best : 0.0;
}

// averages in B (scalar) or B^eps (Euler, rho >= eps and rho e >= eps); NaN fails
template <int PHYS, int DIM>
__device__ __forceinline__ bool admissible(const Params &P, const double *ub) {
    if constexpr (PHYS == PH_EULER) {
        return ub[0] >= P.eps && rho_e<DIM>(ub) >= P.eps;
    } else {
        return ub[0] >= P.lo && ub[0] <= P.hi;
    }
}

// exterior trace on a boundary side (final stage only)
template <int PHYS, int DIM>
__device__ __forceinline__ void boundary_state(const Params &P, int side, const double *ui, double *ue) {
    constexpr int M = ncomp(PHYS, DIM);
    int bc = P.bc[side];
    if (bc == BC_DIRICHLET) {
#pragma unroll
        for (int c = 0; c < M; ++c) ue[c] = P.bcs[side][c];
    } else {
#pragma unroll
        for (int c = 0; c < M; ++c) ue[c] = ui[c];
        if constexpr (PHYS == PH_EULER) {
            if (bc == BC_REFLECT) ue[1 + side / 2] = -ui[1 + side / 2];
        }
    }
}

// Exterior trace of a boundary face point in the final stage: Dirichlet the side's
// state, reflect the interior trace with the normal momentum negated, outflow the
// cell average of the same stage value (avg; a constant state is kept exactly, and
// the Lax--Friedrichs flux keeps its dissipation on outflow faces).
template <int PHYS, int DIM>
__device__ __forceinline__ void exterior_state(const Params &P, int side, const double *ui, const double *avg,
                                               double *ue) {
    constexpr int M = ncomp(PHYS, DIM);
    if (P.bc[side] == BC_OUTFLOW) {
#pragma unroll
        for (int c = 0; c < M; ++c) ue[c] = avg[c];
    } else {
        boundary_state<PHYS, DIM>(P, side, ui, ue);
    }
}

// neighbour across side (0 L, 1 R, 2 B, 3 T), or -1 on a non-periodic boundary
__device__ __forceinline__ int neighbour(const Params &P, int cell, int side) {
    int cx = cell % P.nx, cy = cell / P.nx;
    switch (side) {
    case 0: return cx > 0 ? cell - 1 : (P.bc[0] == BC_PERIODIC ? cell + P.nx - 1 : -1);
    case 1: return cx < P.nx - 1 ? cell + 1 : (P.bc[1] == BC_PERIODIC ? cell - P.nx + 1 : -1);
    case 2: return cy > 0 ? cell - P.nx : (P.bc[2] == BC_PERIODIC ? cell + (P.ny - 1) * P.nx : -1);
    default: return cy < P.ny - 1 ? cell + P.nx : (P.bc[3] == BC_PERIODIC ? cell - (P.ny - 1) * P.nx : -1);
    }
}

// The same, and -1 on a side that a non-rectangular domain's geometry word gives a boundary
// kind (the FP64 final stage; the kernels that reject a geometry keep the plain rule)
__device__ __forceinline__ int neighbour_geo(const Params &P, int cell, int side) {
    if (P.geo != nullptr && ((P.geo[cell] >> (4 * side)) & 15u) != GEO_MESH) return -1;
    return neighbour(P, cell, side);
}

// Exterior trace of a boundary face point of a non-rectangular domain (Examples 4.8, 4.9) in
// the final stage: the side's kind in the cell's geometry word decides.  pos is the face
// point's index along the face, stage the traced stage (its time t0 + c_i dt moves the
// shock line); kind GEO_MESH falls back to the rectangle side's condition.
template <int PHYS, int DIM, int N>
__device__ __forceinline__ void geo_exterior(const Params &P, int cell, int side, int pos, int stage,
                                             const double *ui, const double *avg, double *ue) {
    constexpr int M = ncomp(PHYS, DIM);
    const unsigned kind = (P.geo[cell] >> (4 * side)) & 15u;
    if (kind == GEO_STATE_A || kind == GEO_STATE_B || kind == GEO_SHOCK) {
        int which = kind == GEO_STATE_B ? 1 : 0;
        if (kind == GEO_SHOCK) {
            const NodalTables &T = c_tab[N - 2];
            const int cx = cell % P.nx;
            const double xi = side == 0 ? -1.0 : side == 1 ? 1.0 : T.xg[pos];
            const double x = P.x0 + (cx + 0.5 * (xi + 1.0)) * (2.0 / P.rhx);
            double ci = 0.0;
            for (int j = 0; j < stage; ++j) ci += P.A[stage][j];
            which = x < P.shock_x0 + P.shock_speed * (P.t0 + ci * P.dt) ? 0 : 1;
        }
#pragma unroll
        for (int c = 0; c < M; ++c) ue[c] = P.gstate[which][c];
    } else if (kind == GEO_WALL) {
#pragma unroll
        for (int c = 0; c < M; ++c) ue[c] = ui[c];
        if constexpr (PHYS == PH_EULER) ue[1 + side / 2] = -ui[1 + side / 2];
    } else if (kind == GEO_OUTFLOW) {
#pragma unroll
        for (int c = 0; c < M; ++c) ue[c] = avg[c];
    } else {
        exterior_state<PHYS, DIM>(P, side, ui, avg, ue);
    }
}

// ----------------------------------------------------------------------------- block layout

template <int DIM, int N, int PHYS>
struct Cfg {
    static constexpr int D = DIM;
    static constexpr int NP = N;
    static constexpr int PH = PHYS;
    static constexpr int M = ncomp(PHYS, DIM);
    static constexpr int NN = DIM == 2 ? N * N : N;       // nodes per cell
    static constexpr int NF = DIM == 2 ? N : 1;           // quadrature points per face
    static constexpr int NTR = 2 * DIM * NF;              // face points per cell
    static constexpr int L = nlob(N);                     // Gauss--Lobatto points
    static constexpr int NSK = DIM == 2 ? 2 * N * L : L;  // |S_K|
    static constexpr int NCB = cells_per_block(DIM, N);  // cells per block
    static constexpr int NT = NCB * NN;                   // threads per block (multiple of 32)
    static constexpr int PPT = (NSK + NN - 1) / NN;       // S_K points per thread
    static constexpr int FPT = (NTR + NN - 1) / NN;       // face points per thread
};

template <class C>
struct Smem {
    double u[C::NCB][C::M][C::NN];
    union {  // fluxes live inside eval_G only; the FP32 node copies inside the limiter only
        double f[C::D][C::NCB][C::M][C::NN];
        float uf[C::NCB][C::M][C::NN];
    };
    double tf[C::NCB][C::NTR][C::M];
    double avg[C::NCB][C::M];
    union {  // the limiter's reductions and the final kernel's edge speeds never overlap
        unsigned long long red[C::NCB][C::NN][2];  // ordbits keys
        double ts[C::NCB][C::NTR];  // spectral radii of the traces (eval_G of a traced stage)
        double al[C::NCB][C::NTR];
    };
    double th[C::NCB][2];
    int bad[C::NCB];
};

// value of every component at S_K point p of the cell whose nodes are su
template <int DIM, int N, int M, int NN>
__device__ __forceinline__ void sk_eval(const double (&su)[M][NN], int p, double *v) {
    const NodalTables &T = c_tab[N - 2];
    constexpr int L = nlob(N);
    if constexpr (DIM == 1) {
#pragma unroll
        for (int c = 0; c < M; ++c) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < N; ++a) s = fma(T.Igl[p][a], su[c][a], s);
            v[c] = s;
        }
    } else {
        if (p < N * L) {  // (x^GL_alpha, y^G_beta): interpolate along row beta
            int beta = p / L, al = p - beta * L;
#pragma unroll
            for (int c = 0; c < M; ++c) {
                double s = 0.0;
#pragma unroll
                for (int a = 0; a < N; ++a) s = fma(T.Igl[al][a], su[c][beta * N + a], s);
                v[c] = s;
            }
        } else {  // (x^G_beta, y^GL_alpha): interpolate along column beta
            int q = p - N * L;
            int beta = q / L, al = q - beta * L;
#pragma unroll
            for (int c = 0; c < M; ++c) {
                double s = 0.0;
#pragma unroll
                for (int b = 0; b < N; ++b) s = fma(T.Igl[al][b], su[c][b * N + beta], s);
                v[c] = s;
            }
        }
    }
}

// FP32 screen of the limiter.  v: the FP32 interpolation to S_K point p of the FP32
// copies uf of the cell's FP64 node values; e: a bound on |FP64 interpolation - v| per
// component, 4 (n + 3) 2^-24 sum_a |l_a| |uf_a| (the roundings of the nodes and the
// weights to FP32, of the n FP32 and the n FP64 fused multiply-adds: (n + 3) 2^-24 of
// that sum, taken 4 times).
template <int DIM, int N, int M, int NN>
__device__ __forceinline__ void sk_eval_screen(const float (&su)[M][NN], int p, float *v, float *e) {
    const NodalTables &T = c_tab[N - 2];
    constexpr int L = nlob(N);
    constexpr float K = 4.0f * (N + 3) * 5.9604644775390625e-08f;
    int beta = 0, al = p, stride = 1, off = 0;
    if constexpr (DIM == 2) {
        if (p < N * L) {
            beta = p / L;
            al = p - beta * L;
            stride = 1;
            off = beta * N;
        } else {
            const int q = p - N * L;
            beta = q / L;
            al = q - beta * L;
            stride = N;
            off = beta;
        }
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
        float s = 0.0f, a = 0.0f;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const float w = T.Iglf[al][k], x = su[c][off + k * stride];
            s = fmaf(w, x, s);
            a = fmaf(fabsf(w), fabsf(x), a);
        }
        v[c] = s;
        e[c] = K * a;
    }
}

// True when the FP32 value v (bound e per component on its distance to the FP64 value)
// proves that the FP64 value lies in the bounds: scalar lo <= v <= hi; Euler rho >= eps
// and rho e = E - |m|^2 / (2 rho) >= eps, with rho e bounded below by
// (E - e_E) - (|m| + e_m)^2 / (2 (rho - e_rho)) less 2^-20 of its magnitudes (the FP32
// rounding of this bound and the FP64 rounding of rho e).  NaN and inf never pass.
template <int PHYS, int DIM>
__device__ __forceinline__ bool screen_point(const Params &P, const float *v, const float *e) {
    if (!P.scr_on) return false;
    if constexpr (PHYS == PH_EULER) {
        constexpr int M = DIM + 2;
        const float rlo = v[0] - e[0];
        if (!(rlo >= P.scr_eps && rlo <= 3.0e38f)) return false;
        float m2 = 0.0f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const float ma = fabsf(v[1 + d]) + e[1 + d];
            m2 = fmaf(ma, ma, m2);
        }
        const float kin = 0.5f * m2 / rlo;
        const float elo = v[M - 1] - e[M - 1];
        const float lb = (elo - kin) - 9.5367431640625e-07f * (fabsf(elo) + kin);
        return lb >= P.scr_eps && lb <= 3.0e38f;
    } else {
        return v[0] - e[0] >= P.scr_lo && v[0] + e[0] <= P.scr_hi;
    }
}

// S_K bound predicate used by the limiter's verification and by the margins
template <int PHYS, int DIM>
__device__ __forceinline__ bool point_ok(const Params &P, const double *v) {
    if constexpr (PHYS == PH_EULER) {
        return v[0] >= P.eps && rho_e<DIM>(v) >= P.eps;
    } else {
        return v[0] >= P.lo && v[0] <= P.hi;
    }
}

// Cell averages of all components (Gauss weights; the mass matrix is exact), block
// collective without a barrier: fn(c, avg_c) is called once per component by one
// thread of the cell.  2D Q^3 Euler (16 nodes, a cell on one half-warp): each
// component is split over 4 lanes of 4 terms and summed by two xor shuffles, 6 FP64
// instructions instead of a 16-term chain on 4 of the 16 lanes.  Otherwise one
// thread per component sums the nodes in order.  All threads of the block must call it.
template <class C, class Fn>
__device__ __forceinline__ void cell_averages(const double (&su)[C::M][C::NN], int node, Fn fn) {
    constexpr int DIM = C::D, N = C::NP, M = C::M, NN = C::NN;
    const NodalTables &T = c_tab[N - 2];
    if constexpr (DIM == 2 && NN == 16 && M == 4) {
        const int c = node >> 2, r = node & 3;
        double s = 0.0;
#pragma unroll
        for (int q = 4 * r; q < 4 * r + 4; ++q) s = fma(T.w2[q], su[c][q], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (r == 0) fn(c, s);
    } else {
        for (int c = node; c < M; c += NN) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < NN; ++q) s = fma(DIM == 2 ? T.w2[q] : T.w1[q], su[c][q], s);
            fn(c, s);
        }
    }
}

// ----------------------------------------------------------------------------- limiter

// Rounding safety of the limiter: every theta below 1 is multiplied by
// (1-2^-40) so the rescaled polynomial lands strictly inside the bound; if the
// re-evaluation on S_K still finds a point outside, the final scaling towards
// the average is multiplied by the retry factors 1-2^-30, 1-2^-20, 1-2^-10, 0.
constexpr double kMargin = 1.0 - 9.094947017729282e-13;
__device__ __forceinline__ double retry_factor(int attempt) {
    switch (attempt) {
    case 1: return 1.0 - 9.313225746154785e-10;
    case 2: return 1.0 - 9.5367431640625e-07;
    case 3: return 1.0 - 0.0009765625;
    default: return 0.0;
    }
}

// Scaling limiter of one stage (Prop. 2.4 scalar, eq. Euler-limiter1/2), block
// collective.  u: this thread's node values (in/out).  pts (with need_pts): on return
// the values at this thread's S_K points of the limited polynomial.  With check_avg the
// admissibility of the cell average sets *B.flag (Sec. 4.1 restart test).
//
// Most cells need no limiting.  An FP32 screen (screen_point, with a bound on its
// distance to the FP64 values) first tests every S_K point and the average; when it
// clears every cell of the block, the FP64 limiter would leave all of them unchanged
// (theta = 1, no flag), and it is skipped: the results are those of the FP64 path.
template <class C>
__device__ void limit_block(const Params &P, const Bufs &B, Smem<C> &S, int lc, int node, bool active,
                            double *u, double (&pts)[C::PPT][C::M], bool check_avg, bool stats,
                            bool need_pts = true) {
    constexpr int DIM = C::D, N = C::NP, PHYS = C::PH;
    constexpr int M = C::M, NN = C::NN, NSK = C::NSK, PPT = C::PPT;
    const NodalTables &T = c_tab[N - 2];

    // 1. publish node values (and FP32 copies for the screen)
#pragma unroll
    for (int c = 0; c < M; ++c) {
        S.u[lc][c][node] = u[c];
        S.uf[lc][c][node] = (float)u[c];
    }
    __syncthreads();
    // 2. cell averages (Gauss weights; the mass matrix is exact); FP32 screen of this
    //    thread's S_K points
    cell_averages<C>(S.u[lc], node, [&](int c, double s) { S.avg[lc][c] = s; });
    bool unsafe = false;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        int p = node + j * NN;
        if (p < NSK) {
            float v[M], e[M];
            sk_eval_screen<DIM, N, M, NN>(S.uf[lc], p, v, e);
            if (!screen_point<PHYS, DIM>(P, v, e)) unsafe = true;
        }
    }
    __syncthreads();
    if (node == 0) {  // the average (FP32 rounding of the FP64 value: 2^-22 of it)
        float v[M], e[M];
#pragma unroll
        for (int c = 0; c < M; ++c) {
            v[c] = (float)S.avg[lc][c];
            e[c] = 2.384185791015625e-07f * fabsf(v[c]);
        }
        if (!screen_point<PHYS, DIM>(P, v, e)) unsafe = true;
    }
    if (!__syncthreads_or(unsafe)) {  // every cell of the block cleared
        if (need_pts) {
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                int p = node + j * NN;
                if (p < NSK) sk_eval<DIM, N, M, NN>(S.u[lc], p, pts[j]);
            }
        }
        return;
    }
    // 3. values at S_K and this thread's extremes (order-preserving integer keys)
    unsigned long long kmin = kKeyPosInf, kmax = kKeyNegInf;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        int p = node + j * NN;
        if (p < NSK) {
            sk_eval<DIM, N, M, NN>(S.u[lc], p, pts[j]);
            if (isnan_bits(pts[j][0])) {
                kmin = kKeyNegInf;  // NaN counts as a violation
            } else {
                unsigned long long k = ordbits(pts[j][0]);
                kmin = umin64(kmin, k);
                kmax = umax64(kmax, k);
            }
        }
    }
    S.red[lc][node][0] = kmin;
    S.red[lc][node][1] = kmax;
    double ub[M];
#pragma unroll
    for (int c = 0; c < M; ++c) ub[c] = S.avg[lc][c];
    __syncthreads();
    // 4. leader: admissibility of the average and theta (theta_1 for Euler)
    double reb = 0.0;  // leader: rho e of the average (Euler)
    if (node == 0) {
        unsigned long long kmn = kKeyPosInf, kmx = kKeyNegInf;
        for (int q = 0; q < NN; ++q) {
            kmn = umin64(kmn, S.red[lc][q][0]);
            kmx = umax64(kmx, S.red[lc][q][1]);
        }
        const double mn = ordbits_inv(kmn), mx = ordbits_inv(kmx);
        if constexpr (PHYS == PH_EULER) {
            reb = rho_e<DIM>(ub);
            if (check_avg && active && !(ge_pos_bits(ub[0], P.eps) && ge_pos_bits(reb, P.eps))) atomicOr(B.flag, 1);
        } else {
            if (check_avg && active && !admissible<PHYS, DIM>(P, ub)) atomicOr(B.flag, 1);
        }
        double th = 1.0;
        if constexpr (PHYS == PH_EULER) {
            if (!ge_pos_bits(mn, P.eps)) th = ratio01(ub[0] - P.eps, ub[0] - mn);
        } else {
            if (mx > P.hi) th = fmin(th, ratio01(P.hi - ub[0], mx - ub[0]));
            if (mn < P.lo) th = fmin(th, ratio01(ub[0] - P.lo, ub[0] - mn));
        }
        S.th[lc][0] = below_one(th) ? th * kMargin : th;
        S.th[lc][1] = 1.0;
        S.bad[lc] = 0;
    }
    __syncthreads();
    double th1 = S.th[lc][0];
    double th2 = 1.0;
    if constexpr (PHYS == PH_EULER) {
        // 5. rho e at S_K with the density already scaled by theta_1
        unsigned long long km = kKeyPosInf, kt = ordbits(1.0);
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            int p = node + j * NN;
            if (p < NSK) {
                double v[M];
#pragma unroll
                for (int c = 0; c < M; ++c) v[c] = pts[j][c];
                if (below_one(th1)) v[0] = th1 * (v[0] - ub[0]) + ub[0];
                double re = rho_e<DIM>(v);
                km = isnan_bits(re) ? kKeyNegInf : umin64(km, ordbits(re));  // NaN counts as a violation
                // the exact solve: the smallest per-point theta over the violating points
                if (P.theta2_exact && !ge_pos_bits(re, P.eps))
                    kt = umin64(kt, ordbits(isnan_bits(re) ? 0.0 : theta2_point<DIM>(ub, v, P.eps)));
            }
        }
        S.red[lc][node][1] = km;
        S.red[lc][node][0] = kt;
        __syncthreads();
        if (node == 0) {
            unsigned long long kmn = kKeyPosInf, ktn = ordbits(1.0);
            for (int q = 0; q < NN; ++q) {
                kmn = umin64(kmn, S.red[lc][q][1]);
                ktn = umin64(ktn, S.red[lc][q][0]);
            }
            const double mn = ordbits_inv(kmn);
            S.th[lc][1] = ge_pos_bits(mn, P.eps) ? 1.0
                          : P.theta2_exact        ? ordbits_inv(ktn) * kMargin
                                                  : ratio01(reb - P.eps, reb - mn) * kMargin;
        }
        __syncthreads();
        th2 = S.th[lc][1];
    }
    // 6. rescale towards the average
    bool limited = below_one(th1) || below_one(th2);
    double uo[M];
#pragma unroll
    for (int c = 0; c < M; ++c) uo[c] = u[c];
    auto apply = [&](double t2) {
        if constexpr (PHYS == PH_EULER) {
            double r = below_one(th1) ? th1 * (uo[0] - ub[0]) + ub[0] : uo[0];
            u[0] = below_one(t2) ? t2 * (r - ub[0]) + ub[0] : r;
#pragma unroll
            for (int c = 1; c < M; ++c) u[c] = below_one(t2) ? t2 * (uo[c] - ub[c]) + ub[c] : uo[c];
        } else {
            double t = th1 * t2;
            u[0] = t < 1.0 ? t * (uo[0] - ub[0]) + ub[0] : uo[0];
        }
    };
    double tfin = th2;
    if (limited) apply(th2);
    // 7. verify the limited cells on S_K with the same interpolation; shrink on a
    //    rounding violation (the final scaling factor towards the average)
    bool any_limited = __syncthreads_or(limited);
    if (any_limited) {
        for (int attempt = 0; attempt <= 4; ++attempt) {
#pragma unroll
            for (int c = 0; c < M; ++c) S.u[lc][c][node] = u[c];
            __syncthreads();
            bool viol = false;
            if (limited) {
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    int p = node + j * NN;
                    if (p < NSK) {
                        sk_eval<DIM, N, M, NN>(S.u[lc], p, pts[j]);
                        if (!point_ok<PHYS, DIM>(P, pts[j])) viol = true;
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
                // Euler: theta_2 (all components); scalars: th2 == 1 so the factor multiplies theta
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
}

// ----------------------------------------------------------------------------- G

// G(u) at this thread's node (block collective).  trs receives the interior
// trace states of this thread's face points; their normal fluxes stay in S.tf and,
// with want_speed, their spectral radii go to S.ts (both read back by the thread
// that computed them, for the final stage's Lax--Friedrichs flux of traced stages).
template <class C>
__device__ void eval_G(const Params &P, Smem<C> &S, int lc, int node, const double *u, double *g,
                       double (&trs)[C::FPT][C::M], bool want_speed = false) {
    constexpr int DIM = C::D, N = C::NP, PHYS = C::PH;
    constexpr int M = C::M, NN = C::NN, NF = C::NF, NTR = C::NTR, FPT = C::FPT;
    const NodalTables &T = c_tab[N - 2];
    const int a = node % N, b = DIM == 2 ? node / N : 0;
    // 1. flux at the node
    {
        double fx[M], fy[M];
        if constexpr (DIM == 2) {
            flux_xy<PHYS>(P, u, fx, fy);
        } else {
            flux_dir<PHYS, DIM>(P, u, 0, fx);
        }
#pragma unroll
        for (int c = 0; c < M; ++c) {
            S.u[lc][c][node] = u[c];
            S.f[0][lc][c][node] = fx[c];
            if constexpr (DIM == 2) S.f[1][lc][c][node] = fy[c];
        }
    }
    __syncthreads();
    // 2. volume term and interior traces
    double vx[M], vy[M];
#pragma unroll
    for (int c = 0; c < M; ++c) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < N; ++q) s = fma(T.Dhat[a][q], S.f[0][lc][c][b * N + q], s);
        vx[c] = s;
        if constexpr (DIM == 2) {
            double t = 0.0;
#pragma unroll
            for (int r = 0; r < N; ++r) t = fma(T.Dhat[b][r], S.f[1][lc][c][r * N + a], t);
            vy[c] = t;
        }
    }
#pragma unroll
    for (int j = 0; j < FPT; ++j) {
        int fp = node + j * NN;
        if (fp < NTR) {
            int face = fp / NF, pos = fp - face * NF;
            const double *l = (face & 1) ? T.lp : T.lm;
#pragma unroll
            for (int c = 0; c < M; ++c) {
                double s = 0.0;
                if (DIM == 1 || face < 2) {
#pragma unroll
                    for (int q = 0; q < N; ++q) s = fma(l[q], S.u[lc][c][pos * N + q], s);
                } else {
#pragma unroll
                    for (int q = 0; q < N; ++q) s = fma(l[q], S.u[lc][c][q * N + pos], s);
                }
                trs[j][c] = s;
            }
            double f[M];
            const double ri = recip_rho<PHYS>(trs[j]);
            flux_dir_ri<PHYS, DIM>(P, trs[j], face >> 1, ri, f);
#pragma unroll
            for (int c = 0; c < M; ++c) S.tf[lc][fp][c] = f[c];
            if (want_speed) S.ts[lc][fp] = speed_dir_ri<PHYS, DIM>(P, trs[j], face >> 1, ri);
        }
    }
    __syncthreads();
    // 3. lift the interior-trace edge terms
#pragma unroll
    for (int c = 0; c < M; ++c) {
        double gx = vx[c] - T.liftp[a] * S.tf[lc][NF + b][c] + T.liftm[a] * S.tf[lc][b][c];
        double gv = P.rhx * gx;
        if constexpr (DIM == 2) {
            double gy = vy[c] - T.liftp[b] * S.tf[lc][3 * NF + a][c] + T.liftm[b] * S.tf[lc][2 * NF + a][c];
            gv = fma(P.rhy, gy, gv);
        }
        g[c] = gv;
    }
}

// ----------------------------------------------------------------------------- kernels

template <int DIM, int N, int PHYS>
__device__ __forceinline__ void load_node(const Params &P, const double *src, int cell, int node, bool active,
                                          double *u) {
    using C = Cfg<DIM, N, PHYS>;
#pragma unroll
    for (int c = 0; c < C::M; ++c) {
        if (active) {
            u[c] = src[((size_t)c * P.ncell + cell) * C::NN + node];
        } else {  // benign padding state for idle threads of the last block
            u[c] = (PHYS == PH_EULER && (c == 0 || c == C::M - 1)) ? 1.0 : (PHYS == PH_EULER ? 0.0 : 0.5 * (P.lo + P.hi));
        }
    }
}

template <int DIM, int N, int PHYS>
__device__ __forceinline__ void store_node(const Params &P, double *dst, int cell, int node, bool active,
                                           const double *u) {
    using C = Cfg<DIM, N, PHYS>;
    if (!active) return;
#pragma unroll
    for (int c = 0; c < C::M; ++c) dst[((size_t)c * P.ncell + cell) * C::NN + node] = u[c];
}

// Inner stages (cell-local, no neighbour data): for i = 1..s
//   u^(i) = u^n + dt sum_{j<i} a_ij G(u~^(j)),  u~^(i) = L(u^(i))   (eq. rkdg-lim)
// and the accumulation u* = u^n + dt sum_i b_i G(u~^(i)); the traces of every
// u~^(i) with b_i != 0 go to B.tr for the final kernel.
// The L2 projection of this thread's node values onto the total-degree space P^k (2D; a block
// collective): v at node = sum_q pk[node][q] v_q per component, through S.u.
template <class C>
__device__ __forceinline__ void project_pk(Smem<C> &S, int lc, int node, double *v) {
    if constexpr (C::D == 2) {
        constexpr int M = C::M, NN = C::NN;
        const NodalTables &T = c_tab[C::NP - 2];
        __syncthreads();  // earlier readers of S.u are done
#pragma unroll
        for (int c = 0; c < M; ++c) S.u[lc][c][node] = v[c];
        __syncthreads();
#pragma unroll
        for (int c = 0; c < M; ++c) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < NN; ++q) s = fma(T.pk[node][q], S.u[lc][c][q], s);
            v[c] = s;
        }
        __syncthreads();  // S.u is free again
    }
}

// The source of Example 4.2's scenario I, S = d_t U + div F(U) of the manufactured solution
// rho = e^-t sin 2pi(x+y) + 2, w = (e^-t cos 2pi x sin 2pi y + 2, e^-t sin 2pi x cos 2pi y + 2),
// e = e^-t cos 2pi(x+y) / 2 + 1, at (x, y, t).  Each primitive q is held with its t-, x- and
// y-derivatives (q[0..3]); products by the product rule, then the four balance laws.
__device__ inline void scenario1_source(double gamma, double x, double y, double t, double *S) {
    const double w = 6.283185307179586, a = exp(-t);
    double sxy, cxy, sx, cx, sy, cy;
    sincos(w * (x + y), &sxy, &cxy);
    sincos(w * x, &sx, &cx);
    sincos(w * y, &sy, &cy);
    const double rho[4] = {a * sxy + 2.0, -a * sxy, w * a * cxy, w * a * cxy};
    const double vx[4] = {a * cx * sy + 2.0, -a * cx * sy, -w * a * sx * sy, w * a * cx * cy};
    const double vy[4] = {a * sx * cy + 2.0, -a * sx * cy, w * a * cx * cy, -w * a * sx * sy};
    const double ei[4] = {0.5 * a * cxy + 1.0, -0.5 * a * cxy, -0.5 * w * a * sxy, -0.5 * w * a * sxy};
    auto prod = [](const double *f, const double *g, double *h) {  // h = f g with its derivatives
        h[0] = f[0] * g[0];
#pragma unroll
        for (int d = 1; d < 4; ++d) h[d] = f[d] * g[0] + f[0] * g[d];
    };
    double mx[4], my[4], re[4], mxx[4], mxy[4], myy[4], kx[4], ky[4];
    prod(rho, vx, mx);   // rho w_x
    prod(rho, vy, my);   // rho w_y
    prod(rho, ei, re);   // rho e
    prod(mx, vx, mxx);   // rho w_x^2
    prod(mx, vy, mxy);   // rho w_x w_y
    prod(my, vy, myy);   // rho w_y^2
    double E[4], H[4], p[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        p[d] = (gamma - 1.0) * re[d];
        E[d] = re[d] + 0.5 * (mxx[d] + myy[d]);
        H[d] = E[d] + p[d];  // E + p
    }
    prod(H, vx, kx);  // (E + p) w_x
    prod(H, vy, ky);  // (E + p) w_y
    // index 1: d/dt, 2: d/dx, 3: d/dy
    S[0] = rho[1] + mx[2] + my[3];
    S[1] = mx[1] + mxx[2] + p[2] + mxy[3];
    S[2] = my[1] + mxy[2] + myy[3] + p[3];
    S[3] = E[1] + kx[2] + ky[3];
}

// G += S at this thread's node for stage i (time t0 + c_i dt, c_i the row sum of A): the
// collocated source is its projection by the (k+1)-point Gauss rule.
template <int DIM, int N, int PHYS>
__device__ __forceinline__ void add_source(const Params &P, int cell, int node, int stage, double *g) {
    if constexpr (DIM == 2 && PHYS == PH_EULER) {
        const NodalTables &T = c_tab[N - 2];
        double c = 0.0;
        for (int j = 0; j < stage; ++j) c += P.A[stage][j];
        const int cx = cell % P.nx, cy = cell / P.nx;
        const int a = node % N, b = node / N;
        const double hx = 2.0 / P.rhx, hy = 2.0 / P.rhy;
        const double x = P.x0 + (cx + 0.5 * (T.xg[a] + 1.0)) * hx;
        const double y = P.y0 + (cy + 0.5 * (T.xg[b] + 1.0)) * hy;
        double src[4];
        scenario1_source(P.gamma, x, y, P.t0 + c * P.dt, src);
#pragma unroll
        for (int k = 0; k < 4; ++k) g[k] += src[k];
    }
}

template <int DIM, int N, int PHYS>
__device__ __forceinline__ void inner_body(const Params &P, const Bufs &B, int blk) {
    using C = Cfg<DIM, N, PHYS>;
    constexpr int M = C::M, NN = C::NN, NTR = C::NTR, FPT = C::FPT;
    __shared__ Smem<C> S;
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blk * C::NCB + lc;
    const bool active = cell < P.ncell;
    const bool own = active && owned(P, cell) && !solid_cell(P, cell);  // counts in the flag and statistics
    double un[M], cur[M], acc[M], gh[MAXS][M];
    load_node<DIM, N, PHYS>(P, B.un, cell, node, active, un);
#pragma unroll
    for (int c = 0; c < M; ++c) cur[c] = acc[c] = un[c];
#pragma unroll
    for (int i = 0; i < MAXS; ++i) {
        if (i >= P.s) break;
        if (i > 0) {
#pragma unroll
            for (int c = 0; c < M; ++c) {
                double v = un[c];
#pragma unroll
                for (int j = 0; j < i; ++j)
                    if (nonzero_bits(P.A[i][j])) v = fma(P.dt * P.A[i][j], gh[j][c], v);
                cur[c] = v;
            }
            if (P.pk) project_pk<C>(S, lc, node, cur);
            double pts[C::PPT][M];
            limit_block(P, B, S, lc, node, own, cur, pts, true, true, false);
        }
        double trs[FPT][M];
        const bool keep_faces = P.slot[i] >= 0 && B.tfs != nullptr;
        eval_G(P, S, lc, node, cur, gh[i], trs, keep_faces);
        if (P.source && active) add_source<DIM, N, PHYS>(P, cell, node, i, gh[i]);
        if (P.slot[i] >= 0) {  // cell average of the traced stage value (outflow exterior state)
            const NodalTables &T = c_tab[N - 2];
            cell_averages<C>(S.u[lc], node, [&](int c, double s) {
                if (active) B.tavg[((size_t)P.slot[i] * M + c) * P.ncell + cell] = s;
            });
            __syncthreads();
        }
        if (P.mode == MODE_OP_G) {
#pragma unroll
            for (int c = 0; c < M; ++c) acc[c] = gh[i][c];
        } else if (nonzero_bits(P.b[i])) {
#pragma unroll
            for (int c = 0; c < M; ++c) acc[c] = fma(P.dt * P.b[i], gh[i][c], acc[c]);
        }
        if (P.slot[i] >= 0 && active) {
            double *dst = B.tr + (size_t)P.slot[i] * M * P.ncell * NTR;
            double *dfs = keep_faces ? B.tfs + (size_t)P.slot[i] * (M + 1) * P.ncell * NTR : nullptr;
#pragma unroll
            for (int j = 0; j < FPT; ++j) {
                int fp = node + j * NN;
                if (fp < NTR) {
#pragma unroll
                    for (int c = 0; c < M; ++c) dst[((size_t)c * P.ncell + cell) * NTR + fp] = trs[j][c];
                    if (keep_faces) {  // this thread's own entries of S.tf and S.ts
#pragma unroll
                        for (int c = 0; c < M; ++c) dfs[((size_t)c * P.ncell + cell) * NTR + fp] = S.tf[lc][fp][c];
                        dfs[((size_t)M * P.ncell + cell) * NTR + fp] = S.ts[lc][fp];
                    }
                }
            }
        }
    }
    if (P.pk) project_pk<C>(S, lc, node, acc);
    if (active && solid_cell(P, cell))  // outside the domain: G = 0, u* = u^n
#pragma unroll
        for (int c = 0; c < M; ++c) acc[c] = P.mode == MODE_OP_G ? 0.0 : un[c];
    store_node<DIM, N, PHYS>(P, B.ustar, cell, node, active, acc);
}

template <int DIM, int N, int PHYS>
__global__ void __launch_bounds__(Cfg<DIM, N, PHYS>::NT) k_inner(Params P, Bufs B) {
    inner_body<DIM, N, PHYS>(P, B, blockIdx.x);
}

// Final stage: u^{n+1} = u* + dt lift( sum_i b_i (fhat^(i) - f(u_int^(i))) ), then the
// limiter, the admissibility test and a0 of the new state.  Each face flux is
// evaluated from the same ordered pair (lower side, upper side) by both cells
// sharing the face, so the update is conservative to round-off.
template <int DIM, int N, int PHYS, bool STORED = false>
__device__ __forceinline__ void final_body(const Params &P, const Bufs &B, int blk) {
    using C = Cfg<DIM, N, PHYS>;
    constexpr int M = C::M, NN = C::NN, NF = C::NF, NTR = C::NTR, FPT = C::FPT;
    __shared__ Smem<C> S;
    const NodalTables &T = c_tab[N - 2];
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blk * C::NCB + lc;
    const bool active = cell < P.ncell;
    const bool own = active && owned(P, cell) && !solid_cell(P, cell);  // counts in the flag, statistics and rate
    const int a = node % N, b = DIM == 2 ? node / N : 0;
    double u[M];
    load_node<DIM, N, PHYS>(P, B.ustar, cell, node, active, u);

    double dc[FPT][M];
#pragma unroll
    for (int j = 0; j < FPT; ++j)
#pragma unroll
        for (int c = 0; c < M; ++c) dc[j][c] = 0.0;

    for (int i = 0; i < P.s; ++i) {
        if (P.slot[i] < 0) continue;
        const double *tr = B.tr + (size_t)P.slot[i] * M * P.ncell * NTR;
        // fluxes and spectral radii of interior traces: as the inner kernel stored them
        // (STORED, B.tfs), else recomputed here; the exterior state of a boundary face
        // always here
        const double *tfs = STORED ? B.tfs + (size_t)P.slot[i] * (M + 1) * P.ncell * NTR : nullptr;
        double ui[FPT][M], ue[FPT][M], riI[FPT], riE[FPT];
        int nbr[FPT];
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            int fp = node + j * NN;
            nbr[j] = -1;
            if (fp < NTR && active) {
                int face = fp / NF, pos = fp - face * NF;
#pragma unroll
                for (int c = 0; c < M; ++c) ui[j][c] = tr[((size_t)c * P.ncell + cell) * NTR + fp];
                int nb = neighbour_geo(P, cell, face);
                nbr[j] = nb;
                int ofp = (face ^ 1) * NF + pos;
                if (nb >= 0) {
#pragma unroll
                    for (int c = 0; c < M; ++c) ue[j][c] = tr[((size_t)c * P.ncell + nb) * NTR + ofp];
                } else {
                    double av[M];
#pragma unroll
                    for (int c = 0; c < M; ++c) av[c] = B.tavg[((size_t)P.slot[i] * M + c) * P.ncell + cell];
                    if (P.geo != nullptr)
                        geo_exterior<PHYS, DIM, N>(P, cell, face, pos, i, ui[j], av, ue[j]);
                    else
                        exterior_state<PHYS, DIM>(P, face, ui[j], av, ue[j]);
                }
                int dir = face >> 1;
                double sI, sE;
                if constexpr (STORED) {
                    sI = tfs[((size_t)M * P.ncell + cell) * NTR + fp];
                    if (nb >= 0) {
                        sE = tfs[((size_t)M * P.ncell + nb) * NTR + ofp];
                    } else {
                        riE[j] = recip_rho<PHYS>(ue[j]);
                        sE = speed_dir_ri<PHYS, DIM>(P, ue[j], dir, riE[j]);
                    }
                } else {
                    riI[j] = recip_rho<PHYS>(ui[j]);
                    riE[j] = recip_rho<PHYS>(ue[j]);
                    sI = speed_dir_ri<PHYS, DIM>(P, ui[j], dir, riI[j]);
                    sE = speed_dir_ri<PHYS, DIM>(P, ue[j], dir, riE[j]);
                }
                S.al[lc][fp] = fmax_nonneg(sI, sE);
            } else if (fp < NTR) {
                S.al[lc][fp] = 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            int fp = node + j * NN;
            if (fp < NTR && active) {
                int face = fp / NF, pos = fp - face * NF;
                int dir = face >> 1;
                double alpha = 0.0;  // per-edge LF viscosity: max over the edge's points
#pragma unroll
                for (int q = 0; q < NF; ++q) alpha = fmax_nonneg(alpha, S.al[lc][face * NF + q]);
                double fI[M], fE[M];
                const int nb = nbr[j];
                if constexpr (STORED) {
#pragma unroll
                    for (int c = 0; c < M; ++c) fI[c] = tfs[((size_t)c * P.ncell + cell) * NTR + fp];
                    if (nb >= 0) {
                        const int ofp = (face ^ 1) * NF + pos;
#pragma unroll
                        for (int c = 0; c < M; ++c) fE[c] = tfs[((size_t)c * P.ncell + nb) * NTR + ofp];
                    } else {
                        flux_dir_ri<PHYS, DIM>(P, ue[j], dir, riE[j], fE);
                    }
                } else {
                    flux_dir_ri<PHYS, DIM>(P, ui[j], dir, riI[j], fI);
                    flux_dir_ri<PHYS, DIM>(P, ue[j], dir, riE[j], fE);
                }
                bool upper = face & 1;  // R or T: the cell is on the lower side of the face
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const double uLc = upper ? ui[j][c] : ue[j][c], uRc = upper ? ue[j][c] : ui[j][c];
                    const double fLc = upper ? fI[c] : fE[c], fRc = upper ? fE[c] : fI[c];
                    double fhat = 0.5 * (fLc + fRc) - 0.5 * alpha * (uRc - uLc);
                    dc[j][c] = fma(P.b[i], fhat - fI[c], dc[j][c]);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < FPT; ++j) {
        int fp = node + j * NN;
        if (fp < NTR)
#pragma unroll
            for (int c = 0; c < M; ++c) S.tf[lc][fp][c] = dc[j][c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < M; ++c) {
        double cx = -T.liftp[a] * S.tf[lc][NF + b][c] + T.liftm[a] * S.tf[lc][b][c];
        double corr = P.rhx * cx;
        if constexpr (DIM == 2) {
            double cy = -T.liftp[b] * S.tf[lc][3 * NF + a][c] + T.liftm[b] * S.tf[lc][2 * NF + a][c];
            corr = fma(P.rhy, cy, corr);
        }
        u[c] = fma(P.dt, corr, u[c]);
    }
    if (P.pk) project_pk<C>(S, lc, node, u);
    if (P.mode == MODE_OP_F) {
        if (active && solid_cell(P, cell))  // outside the domain: no operator
#pragma unroll
            for (int c = 0; c < M; ++c) u[c] = 0.0;
        store_node<DIM, N, PHYS>(P, B.unew, cell, node, active, u);
        return;
    }
    if (P.defer_limit) {  // averages and their admissibility here; limiters in k_trouble
#pragma unroll
        for (int c = 0; c < M; ++c) S.u[lc][c][node] = u[c];
        __syncthreads();
        cell_averages<C>(S.u[lc], node, [&](int c, double s) {
            S.avg[lc][c] = s;
            if (active) B.aux[(size_t)cell * M + c] = s;
        });
        __syncthreads();
        if (node == 0 && own && !admissible<PHYS, DIM>(P, S.avg[lc])) atomicOr(B.flag, 1);
        store_node<DIM, N, PHYS>(P, B.unew, cell, node, active, u);
        return;
    }
    double pts[C::PPT][M];
    limit_block(P, B, S, lc, node, own, u, pts, true, true);
    // wave-speed rate of the new state over its S_K points (next trial step)
    double amax = 0.0;
#pragma unroll
    for (int j = 0; j < C::PPT; ++j) {
        int p = node + j * NN;
        if (p < C::NSK && own) amax = fmax_nonneg(amax, sk_rate<PHYS, DIM>(P, pts[j]));
    }
    unsigned long long abits = dbits(amax);  // non-negative: the bits order as the values
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) abits = umax64(abits, __shfl_xor_sync(0xffffffffu, abits, o));
    if ((threadIdx.x & 31) == 0 && abits > 0ull) atomicMax(B.a0, abits);
    if (active && solid_cell(P, cell)) load_node<DIM, N, PHYS>(P, B.un, cell, node, true, u);  // keeps u^n
    store_node<DIM, N, PHYS>(P, B.unew, cell, node, active, u);
}

// Resident blocks per SM the FP64 final kernel's register budget is sized for: two of the
// 2D Q^2 blocks (288 threads), five of the 128-thread ones.  Unbounded, the owned-box test of
// the domain decomposition took the Q^2 kernel from 96 to 126 registers, one resident block,
// and the 1024^2 Q^2 launch from 4.78 to 6.33 ms.
template <class C>
constexpr int fp64_final_min_blocks() {
    return C::NT > 128 ? 2 : 5;
}

template <int DIM, int N, int PHYS, bool STORED>
__global__ void __launch_bounds__(Cfg<DIM, N, PHYS>::NT, fp64_final_min_blocks<Cfg<DIM, N, PHYS>>())
    k_final(Params P, Bufs B) {
    final_body<DIM, N, PHYS, STORED>(P, B, blockIdx.x);
}

// Limiter applied to a state (set-up projection, operator checks): un -> unew.  In
// MODE_RATE it also posts the wave-speed rate of the limited state to B.a0: the
// limiter leaves this thread's S_K values of the final nodal values in pts, the
// same interpolation of the same values that the scan kernel would take.
template <int DIM, int N, int PHYS>
__global__ void __launch_bounds__(Cfg<DIM, N, PHYS>::NT) k_limit(Params P, Bufs B) {
    using C = Cfg<DIM, N, PHYS>;
    __shared__ Smem<C> S;
    const int lc = threadIdx.x / C::NN, node = threadIdx.x - lc * C::NN;
    const int cell = blockIdx.x * C::NCB + lc;
    const bool active = cell < P.ncell;
    const bool own = active && owned(P, cell) && !solid_cell(P, cell);
    const bool rate = P.mode == MODE_RATE || P.mode == MODE_LIMIT_FINAL;
    const bool check = P.mode == MODE_LIMIT_CHECK || P.mode == MODE_LIMIT_FINAL;  // standard RKDG stages
    double u[C::M], pts[C::PPT][C::M];
    load_node<DIM, N, PHYS>(P, B.un, cell, node, active, u);
    if (P.pk) project_pk<C>(S, lc, node, u);  // a state set in P^k: its L2 projection first
    limit_block(P, B, S, lc, node, own, u, pts, check, check, rate);
    if (rate) {
        double amax = 0.0;
#pragma unroll
        for (int j = 0; j < C::PPT; ++j) {
            int p = node + j * C::NN;
            if (p < C::NSK && own) amax = fmax(amax, sk_rate<PHYS, DIM>(P, pts[j]));
        }
        unsigned long long abits = dbits(amax);  // non-negative: the bits order as the values
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) abits = umax64(abits, __shfl_xor_sync(0xffffffffu, abits, o));
        if ((threadIdx.x & 31) == 0 && abits > 0ull) atomicMax(B.a0, abits);
    }
    if (active && solid_cell(P, cell)) load_node<DIM, N, PHYS>(P, B.un, cell, node, true, u);  // not limited
    store_node<DIM, N, PHYS>(P, B.unew, cell, node, active, u);
}

// a0 over the S_K points of un, and the two smallest bound margins.
template <int DIM, int N, int PHYS>
__global__ void __launch_bounds__(Cfg<DIM, N, PHYS>::NT) k_scan(Params P, Bufs B) {
    using C = Cfg<DIM, N, PHYS>;
    constexpr int M = C::M, NN = C::NN;
    __shared__ Smem<C> S;
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blockIdx.x * C::NCB + lc;
    const bool active = cell < P.ncell;
    const bool own = active && owned(P, cell) && !solid_cell(P, cell);
    double u[M];
    load_node<DIM, N, PHYS>(P, B.un, cell, node, active, u);
#pragma unroll
    for (int c = 0; c < M; ++c) S.u[lc][c][node] = u[c];
    __syncthreads();
    double amax = 0.0, m0 = INFINITY, m1 = INFINITY;
    const bool margins = P.mode != MODE_RATE;
#pragma unroll
    for (int j = 0; j < C::PPT; ++j) {
        int p = node + j * NN;
        if (p < C::NSK && own) {
            double v[M];
            sk_eval<DIM, N, M, NN>(S.u[lc], p, v);
            amax = fmax(amax, sk_rate<PHYS, DIM>(P, v));
            if (!margins) continue;
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
    // extremes on the integer units: the rate is non-negative; the margins as ordbits keys
    unsigned long long ab = dbits(amax), k0 = ordbits(m0), k1 = ordbits(m1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ab = umax64(ab, __shfl_xor_sync(0xffffffffu, ab, o));
        if (margins) {
            k0 = umin64(k0, __shfl_xor_sync(0xffffffffu, k0, o));
            k1 = umin64(k1, __shfl_xor_sync(0xffffffffu, k1, o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        if (ab > 0ull) atomicMax(B.a0, ab);
        if (margins) {
            atomicMin(&B.ord[0], k0);
            atomicMin(&B.ord[1], k1);
        }
    }
}

// Cell averages of un -> aux[cell][m]
template <int DIM, int N, int PHYS>
__global__ void k_avg(Params P, Bufs B) {
    using C = Cfg<DIM, N, PHYS>;
    const NodalTables &T = c_tab[N - 2];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.ncell * C::M) return;
    int cell = t / C::M, c = t - cell * C::M;
    const double *u = B.un + ((size_t)c * P.ncell + cell) * C::NN;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < C::NN; ++q) s = fma(DIM == 2 ? T.w2[q] : T.w1[q], u[q], s);
    B.aux[t] = s;
}

// x < 0.0 (false for -0 and NaN)
__device__ __forceinline__ bool negative_bits(double x) {
    const unsigned long long b = dbits(x);
    return b > 0x8000000000000000ull && b <= 0xfff0000000000000ull;
}
// minmod(a, b, c): the argument of least magnitude when all three share one sign, else 0,
// on the integer units (for values of one sign the one of least magnitude has the
// smallest bit pattern)
__device__ __forceinline__ double minmod3_bits(double a, double b, double c) {
    const bool pos = positive_bits(a) && positive_bits(b) && positive_bits(c);
    const bool neg = negative_bits(a) && negative_bits(b) && negative_bits(c);
    return (pos || neg) ? bitsd(umin64(dbits(a), umin64(dbits(b), dbits(c)))) : 0.0;
}
// The TVB-modified minmod test of one face-averaged trace deviation t against the
// neighbour differences dp, dm and the threshold thr: true when minmod changes t, i.e.
// (|t| <= thr ? t : minmod(t, dp, dm)) != t, on the integer units.  thr_ok = thr >= 0.
__device__ __forceinline__ bool tvb_changes(double t, double dp, double dm, double thr, bool thr_ok) {
    constexpr unsigned long long kAbs = 0x7fffffffffffffffull;
    if (thr_ok && (dbits(t) & kAbs) <= (dbits(thr) & kAbs)) return false;
    if (isnan_bits(t)) return true;  // a NaN deviation compares unequal to itself
    const unsigned long long m = dbits(minmod3_bits(t, dp, dm)), tb = dbits(t);
    return m != tb && ((m | tb) << 1) != 0ull;  // +0 and -0 compare equal
}

// Average of component c of the neighbour of `cell` across `side` (the averages are in
// aux, [cell][m]); across a domain boundary, the boundary condition applied to the
// cell's own average.
template <int PHYS, int DIM>
__device__ __forceinline__ double nb_average(const Params &P, const double *aux, int cell, int side, int c) {
    constexpr int M = ncomp(PHYS, DIM);
    const int nb = neighbour(P, cell, side);
    if (nb >= 0) return aux[(size_t)nb * M + c];
    double own[M], ext[M];
#pragma unroll
    for (int i = 0; i < M; ++i) own[i] = aux[(size_t)cell * M + i];
    boundary_state<PHYS, DIM>(P, side, own, ext);
    return ext[c];
}

// Plain troubled-cell indicator and shock limiter, then the scaling limiter (an
// optional anti-oscillation stage outside the paper's method, run once per step
// after the final stage so the inner stages stay compact).  Per component and
// direction: face-averaged trace deviations ut_R = avg_face(u_R) - ubar,
// ut_L = ubar - avg_face(u_L) against D+ / D- of the cell averages (neighbours
// across a boundary follow its condition); the cell is troubled if the
// TVB-modified minmod changes either deviation.  A troubled cell becomes
// ubar + minmod(c_x, D+x, D-x) xi + minmod(c_y, D+y, D-y) eta, with c_x, c_y its
// first Legendre moments.  Reads unew and the averages in aux; writes unew.
template <int DIM, int N, int PHYS>
__device__ __forceinline__ void trouble_body(const Params &P, const Bufs &B, int blk) {
    using C = Cfg<DIM, N, PHYS>;
    constexpr int M = C::M, NN = C::NN;
    __shared__ Smem<C> S;
    __shared__ double sP1[C::NCB][2][M];
    __shared__ int sTr[C::NCB];
    const NodalTables &T = c_tab[N - 2];
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int cell = blk * C::NCB + lc;
    const bool active = cell < P.ncell;
    const int a = node % N, b = DIM == 2 ? node / N : 0;
    double u[M];
    load_node<DIM, N, PHYS>(P, B.unew, cell, node, active, u);
#pragma unroll
    for (int c = 0; c < M; ++c) S.u[lc][c][node] = u[c];
    if (node == 0) sTr[lc] = 0;
    __syncthreads();
    // the (direction, component) pairs are spread over the cell's threads: each takes the
    // decision and the limited first moment of its pairs
    for (int j = node; j < DIM * M && active; j += NN) {
        const int d = j / M, c = j - d * M;
        const double thr = P.thr[d];
        const double own = B.aux[(size_t)cell * M + c];
        const double lo = nb_average<PHYS, DIM>(P, B.aux, cell, 2 * d, c);
        const double hi = nb_average<PHYS, DIM>(P, B.aux, cell, 2 * d + 1, c);
        double fr = 0.0, fl = 0.0, p1 = 0.0;
        for (int q = 0; q < NN; ++q) {
            double v = S.u[lc][c][q];
            if constexpr (DIM == 2) {
                fr = fma(T.trw2[d][0][q], v, fr);
                fl = fma(T.trw2[d][1][q], v, fl);
                p1 = fma(T.pm2[d][q], v, p1);
            } else {
                fr = fma(T.lp[q], v, fr);
                fl = fma(T.lm[q], v, fl);
                p1 = fma(T.pm1[q], v, p1);
            }
        }
        double utR = fr - own, utL = own - fl;
        double dp = hi - own, dm = own - lo;
        const bool thr_ok = thr >= 0.0;
        if (tvb_changes(utR, dp, dm, thr, thr_ok) || tvb_changes(utL, dp, dm, thr, thr_ok)) atomicOr(&sTr[lc], 1);
        sP1[lc][d][c] = minmod3_bits(p1, dp, dm);
    }
    __syncthreads();
    bool troubled = active && (P.ind_stage >= 2 ? B.tflags[cell] != 0 : sTr[lc] != 0);
    if (P.ind_stage == 3 && active) {  // learned flags: p > 0.6 troubled, p < 0.4 smooth, else the plain flag
        const float pr = B.prob[cell];
        troubled = pr > 0.6f ? true : (pr < 0.4f ? false : troubled);
    }
    if (troubled) {
#pragma unroll
        for (int c = 0; c < M; ++c) {
            double v = fma(sP1[lc][0][c], T.xg[a], B.aux[(size_t)cell * M + c]);
            if constexpr (DIM == 2) v = fma(sP1[lc][1][c], T.xg[b], v);
            u[c] = v;
        }
    }
    if (node == 0 && active) {
        if (B.tflags && (P.ind_stage == 0 || P.ind_stage == 3)) B.tflags[cell] = troubled ? 1 : 0;
        if (troubled) atomicAdd(B.ntrb, 1ull);
    }
    double pts[C::PPT][M];
    limit_block(P, B, S, lc, node, active, u, pts, false, true);
    double amax = 0.0;
#pragma unroll
    for (int j = 0; j < C::PPT; ++j) {
        int p = node + j * NN;
        if (p < C::NSK && active) amax = fmax_nonneg(amax, sk_rate<PHYS, DIM>(P, pts[j]));
    }
    unsigned long long abits = dbits(amax);  // non-negative: the bits order as the values
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) abits = umax64(abits, __shfl_xor_sync(0xffffffffu, abits, o));
    if ((threadIdx.x & 31) == 0 && abits > 0ull) atomicMax(B.a0, abits);
    store_node<DIM, N, PHYS>(P, B.unew, cell, node, active, u);
}

template <int DIM, int N, int PHYS>
__global__ void __launch_bounds__(Cfg<DIM, N, PHYS>::NT) k_trouble(Params P, Bufs B) {
    trouble_body<DIM, N, PHYS>(P, B, blockIdx.x);
}

// MLP features of every cell (2D Euler) and the plain indicator's decision (tflags).
// Features, per component: the 3x3 neighbourhood of cell averages (neighbours across a
// boundary follow its condition) minus their mean over den = max(range, M hx hy) +
// 1e-6 max|v|, and the cell's first Legendre moments over the same den.  Layout
// [cell][44]: 36 normalised averages ([comp][9], row-major, centre 4), then 8
// normalised moments ([comp][x, y]).  Reads unew and the averages in aux.
// The 36 stencil features of a 2D Euler cell (per component the 3x3 averages minus their
// mean, times scale = 1 / (max(range, M hx hy) + 1e-6 max|v|)) from the cell averages
// aux[cell][m]; v receives the stencil averages and scale the per-component factor.
template <int PHYS>
__device__ __forceinline__ void stencil_features(const Params &P, const double *aux, int cell, float *f,
                                                 double (&v)[9][ncomp(PHYS, 2)], double (&scale)[ncomp(PHYS, 2)]) {
    constexpr int DIM = 2, M = ncomp(PHYS, 2);
    // 3x3 stencil; a position outside the domain takes the nearest in-domain cell's
    // average with the boundary state of each crossed side applied (x side first)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            int cx = cell;
            bool xout = false, yout = false;
            if (dx != 0) {
                int nb = neighbour(P, cell, dx < 0 ? 0 : 1);
                if (nb >= 0) cx = nb; else xout = true;
            }
            int cy = cx;
            if (dy != 0) {
                int nb = neighbour(P, cx, dy < 0 ? 2 : 3);
                if (nb >= 0) cy = nb; else yout = true;
            }
            double val[M], tmp[M];
#pragma unroll
            for (int c = 0; c < M; ++c) val[c] = aux[(size_t)cy * M + c];
            if (xout) {
                boundary_state<PHYS, DIM>(P, dx < 0 ? 0 : 1, val, tmp);
#pragma unroll
                for (int c = 0; c < M; ++c) val[c] = tmp[c];
            }
            if (yout) {
                boundary_state<PHYS, DIM>(P, dy < 0 ? 2 : 3, val, tmp);
#pragma unroll
                for (int c = 0; c < M; ++c) val[c] = tmp[c];
            }
#pragma unroll
            for (int c = 0; c < M; ++c) v[(dy + 1) * 3 + (dx + 1)][c] = val[c];
        }
    // per component: (v - mean) / den and slopes / den, den = max(range, M hx hy) + 1e-6 max|v|
    const double thr = P.thr_feat;
#pragma unroll
    for (int c = 0; c < M; ++c) {
        double mean = 0.0;
        unsigned long long kmx = kKeyNegInf, kmn = kKeyPosInf, kab = 0ull;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            mean += v[q][c];
            if (!isnan_bits(v[q][c])) {  // fmax / fmin ignore NaN
                const unsigned long long k = ordbits(v[q][c]);
                kmx = umax64(kmx, k);
                kmn = umin64(kmn, k);
                kab = umax64(kab, dbits(v[q][c]) & 0x7fffffffffffffffull);
            }
        }
        const double mx = ordbits_inv(kmx), mn = ordbits_inv(kmn), amax = bitsd(kab);
        mean /= 9.0;
        scale[c] = recip_nr(fmax(mx - mn, thr) + (1e-6 * amax + 1e-30));
#pragma unroll
        for (int q = 0; q < 9; ++q) f[c * 9 + q] = (float)((v[q][c] - mean) * scale[c]);
    }
}

template <int DIM, int N, int PHYS>
__device__ __forceinline__ void features_body(const Params &P, const Bufs &B, int blk) {
    constexpr int M = ncomp(PHYS, DIM);
    constexpr int NN = DIM == 2 ? N * N : N;
    const int cell = blk * blockDim.x + threadIdx.x;
    if constexpr (DIM != 2 || PHYS != PH_EULER) {
        return;
    } else {
        if (cell >= P.ncell) return;
        const NodalTables &T = c_tab[N - 2];
        double v[9][M], scale[M];
        stencil_features<PHYS>(P, B.aux, cell, B.feat + (size_t)cell * 44, v, scale);
        float *f = B.feat + (size_t)cell * 44;
#pragma unroll
        for (int c = 0; c < M; ++c) {
            const double *u = B.unew + ((size_t)c * P.ncell + cell) * NN;
            double cx = 0.0, cy = 0.0;
#pragma unroll
            for (int q = 0; q < NN; ++q) {
                int qa = q % N, qb = q / N;
                double w = T.mom2[q] * u[q];
                cx = fma(w, T.xg[qa], cx);
                cy = fma(w, T.xg[qb], cy);
            }
            f[36 + 2 * c] = (float)(cx * scale[c]);
            f[37 + 2 * c] = (float)(cy * scale[c]);
        }
        // the plain indicator's decision for this cell, with the troubled-cell kernel's
        // arithmetic: the label of harvested features and the fallback of the learned flags
        int trouble = 0;
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const double thr = P.thr[d];
            const double *lo = v[d == 0 ? 3 : 1], *hi = v[d == 0 ? 5 : 7], *own = v[4];
            const bool thr_ok = thr >= 0.0;
#pragma unroll
            for (int c = 0; c < M; ++c) {
                const double *uc = B.unew + ((size_t)c * P.ncell + cell) * NN;
                double fr = 0.0, fl = 0.0;
                for (int q = 0; q < NN; ++q) {
                    double val = uc[q];
                    fr = fma(T.trw2[d][0][q], val, fr);
                    fl = fma(T.trw2[d][1][q], val, fl);
                }
                double utR = fr - own[c], utL = own[c] - fl;
                double dp = hi[c] - own[c], dm = own[c] - lo[c];
                if (tvb_changes(utR, dp, dm, thr, thr_ok) || tvb_changes(utL, dp, dm, thr, thr_ok)) trouble = 1;
            }
        }
        if (B.tflags) B.tflags[cell] = trouble;
    }
}

template <int DIM, int N, int PHYS>
__global__ void k_features(Params P, Bufs B) {
    features_body<DIM, N, PHYS>(P, B, blockIdx.x);
}

template <int DIM, int N, int PHYS>
cudaError_t launch_one(int kernel, int nblocks, cudaStream_t st, const Params &P, const Bufs &B) {
    using C = Cfg<DIM, N, PHYS>;
    switch (kernel) {
    case K_INNER: k_inner<DIM, N, PHYS><<<nblocks, C::NT, 0, st>>>(P, B); break;
    case K_FINAL:
        if (B.tfs)
            k_final<DIM, N, PHYS, true><<<nblocks, C::NT, 0, st>>>(P, B);
        else
            k_final<DIM, N, PHYS, false><<<nblocks, C::NT, 0, st>>>(P, B);
        break;
    case K_LIMIT: k_limit<DIM, N, PHYS><<<nblocks, C::NT, 0, st>>>(P, B); break;
    case K_TROUBLE: k_trouble<DIM, N, PHYS><<<nblocks, C::NT, 0, st>>>(P, B); break;
    case K_FEATURES: k_features<DIM, N, PHYS><<<(P.ncell + 127) / 128, 128, 0, st>>>(P, B); break;
    case K_A0:
    case K_MARGINS: k_scan<DIM, N, PHYS><<<nblocks, C::NT, 0, st>>>(P, B); break;
    case K_AVG: {
        int tot = P.ncell * C::M;
        k_avg<DIM, N, PHYS><<<(tot + 255) / 256, 256, 0, st>>>(P, B);
        break;
    }
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int DIM>
cudaError_t launch_dim(int kernel, int n, int phys, int nblocks, cudaStream_t st, const Params &P,
                       const Bufs &B) {
#define CRKDG_CASE(NV, PV) \
    if (n == NV && phys == PV) return launch_one<DIM, NV, PV>(kernel, nblocks, st, P, B);
    CRKDG_CASE(2, PH_ADV) CRKDG_CASE(2, PH_BURG) CRKDG_CASE(2, PH_EULER)
    CRKDG_CASE(3, PH_ADV) CRKDG_CASE(3, PH_BURG) CRKDG_CASE(3, PH_EULER)
    CRKDG_CASE(4, PH_ADV) CRKDG_CASE(4, PH_BURG) CRKDG_CASE(4, PH_EULER)
#undef CRKDG_CASE
    return cudaErrorInvalidValue;
}

}  // namespace crkdg
