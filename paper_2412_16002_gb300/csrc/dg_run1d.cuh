// dg_run1d.cuh -- device-resident step loop for 1D meshes (one persistent
// cooperative launch runs many limited cRKDG steps).
//
// Small 1D problems (a few thousand cells) finish a step in a few microseconds
// of FP64 work, less than a host round trip.  Here one launch keeps the whole
// Sec. 4.1 loop on the device: every block owns chunks of NCB-2 consecutive
// cells plus one halo cell on each side, recomputes the (cell-local) inner
// stages of the halo cells itself, so the final stage's Lax--Friedrichs fluxes
// need no neighbour data from other blocks (compactness, Sec. 1), and only one
// grid barrier per attempt decides acceptance, restart (dt halved) and the next
// trial step from the global admissibility flag and wave-speed rate.
#pragma once

#include "dg_core.cuh"

namespace crkdg {

template <int N, int PHYS, int NCBV>
struct RunCfg1D {
    static constexpr int D = 1;
    static constexpr int NP = N;
    static constexpr int PH = PHYS;
    static constexpr int M = ncomp(PHYS, 1);
    static constexpr int NN = N;
    static constexpr int NF = 1;
    static constexpr int NTR = 2;
    static constexpr int L = nlob(N);
    static constexpr int NSK = L;
    static constexpr int NCB = NCBV;  // cells per chunk including the two halo cells
    static constexpr int NT = NCB * NN;
    static constexpr int PPT = (NSK + NN - 1) / NN;
    static constexpr int FPT = (NTR + NN - 1) / NN;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier on a counter that only grows: every block adds one per
// barrier and waits until the count reaches `target` (the number of arrivals due
// by the end of this barrier), so no block resets anything and the last arrival
// wakes the others by its own add.  The fence before the add publishes the
// block's writes (ordered before it by the block barrier); the acquire load
// orders the reads after it.  The waiting thread then reads the attempt's
// admissibility flag, rate and limited-cell count together (one round trip)
// and hands them to the block.  Bounded wait (2 s of %globaltimer): returns false
// when it expired, and the caller then leaves its step loop.
struct SlotRead {
    int flag;
    unsigned long long rate, nlim;
};
__device__ bool grid_barrier(RunCtl *R, unsigned target, const RunSlot *SL, SlotRead &out) {
    __shared__ int s_ok;
    __shared__ SlotRead s_rd;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(&R->bar_count) : "memory");
        const unsigned long long t0 = global_ns();
        for (;;) {
            unsigned c;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(&R->bar_count) : "memory");
            if ((int)(c - target) >= 0) break;  // wrap-safe: the count never runs 2^31 ahead
            if (global_ns() - t0 > 2000000000ull) {
                ok = 0;
                break;
            }
            __nanosleep(40);
        }
        s_rd.flag = *(const volatile int *)&SL->flag;
        s_rd.rate = *(const volatile unsigned long long *)&SL->rate;
        s_rd.nlim = *(const volatile unsigned long long *)&SL->nlim;
        s_ok = ok;
    }
    __syncthreads();
    out = s_rd;
    return s_ok != 0;
}

template <int N, int PHYS, int NCBV>
__global__ void __launch_bounds__(RunCfg1D<N, PHYS, NCBV>::NT) k_run1d(Params P, double *U0, double *U1,
                                                                        RunCtl *R, int cown) {
    using C = RunCfg1D<N, PHYS, NCBV>;
    constexpr int M = C::M, NN = C::NN;
    const int COWN = cown;  // own cells per chunk (1 .. NCB - 2); slots beyond COWN + 1 stay idle
    __shared__ Smem<C> S;
    __shared__ double sTr[MAXS][C::NCB][2][M];
    __shared__ double sAv[MAXS][C::NCB][M];  // cell averages of the traced stage values
    __shared__ double sFc[MAXS][C::NCB][2][M];  // per face: fhat - f(u_L), fhat - f(u_R)
    __shared__ double sTf[MAXS][C::NCB][2][M];  // normal fluxes of the traces
    __shared__ double sSp[MAXS][C::NCB][2];     // spectral radii of the traces
    const NodalTables &T = c_tab[N - 2];
    const int lc = threadIdx.x / NN, node = threadIdx.x - lc * NN;
    const int a = node;
    const int nchunks = (P.ncell + COWN - 1) / COWN;
    const bool periodic = P.bc[0] == BC_PERIODIC;

    double t = R->t;
    const double t_end = R->t_end, cfl = R->cfl;
    const int nsteps = R->nsteps, maxh = R->max_halvings;
    int cur = R->cur, steps = 0, restarts = 0, halv = 0, it = 0, status = RUN_OK;
    unsigned long long nlim_total = 0;
    double rate_last = -1.0;
    double dt_try = fmin(R->dt0, t_end - t);

    while (steps < nsteps && t < t_end) {
        RunSlot *SL = &R->slot[it % 3];
        Bufs B;
        B.flag = &SL->flag;
        B.nlim = &SL->nlim;
        B.thmin = &SL->thmin;
        B.a0 = &SL->rate;
        const double *un = cur ? U1 : U0;
        double *unew = cur ? U0 : U1;
        const double dt = dt_try;

        for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
            const int c0 = chunk * COWN;        // first own cell of the chunk
            const int graw = c0 - 1 + lc;       // unwrapped global index of this slot
            const bool exists = lc <= COWN + 1 && (periodic || (graw >= 0 && graw < P.ncell));
            const int gc = periodic ? (graw % P.ncell + P.ncell) % P.ncell : graw;
            const bool own = lc >= 1 && lc <= COWN && graw < P.ncell;
            double u0[M], cur_u[M], acc[M], gh[MAXS][M];
            load_node<1, N, PHYS>(P, un, gc, node, exists, u0);
#pragma unroll
            for (int c = 0; c < M; ++c) cur_u[c] = acc[c] = u0[c];
            // inner stages of every cell of the chunk, halo included
#pragma unroll
            for (int i = 0; i < MAXS; ++i) {
                if (i >= P.s) break;
                if (i > 0) {
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        double v = u0[c];
#pragma unroll
                        for (int j = 0; j < i; ++j)
                            if (nonzero_bits(P.A[i][j])) v = fma(dt * P.A[i][j], gh[j][c], v);
                        cur_u[c] = v;
                    }
                    double pts[C::PPT][M];
                    limit_block(P, B, S, lc, node, own, cur_u, pts, true, true, false);
                }
                double trs[C::FPT][M];
                const bool traced = P.slot[i] >= 0;
                eval_G(P, S, lc, node, cur_u, gh[i], trs, traced);
                if (nonzero_bits(P.b[i])) {
#pragma unroll
                    for (int c = 0; c < M; ++c) acc[c] = fma(dt * P.b[i], gh[i][c], acc[c]);
                }
                if (traced && node < 2) {
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        sTr[P.slot[i]][lc][node][c] = trs[0][c];
                        sTf[P.slot[i]][lc][node][c] = S.tf[lc][node][c];  // written by this thread
                    }
                    sSp[P.slot[i]][lc][node] = S.ts[lc][node];
                }
                if (P.slot[i] >= 0) {  // S.u holds the stage values until the next stage's limiter
                    for (int c = node; c < M; c += NN) {
                        double s = 0.0;
#pragma unroll
                        for (int q = 0; q < NN; ++q) s = fma(T.w1[q], S.u[lc][c][q], s);
                        sAv[P.slot[i]][lc][c] = s;
                    }
                    __syncthreads();
                }
            }
            __syncthreads();
            // final stage: Lax--Friedrichs flux of every face of the chunk and every traced
            // stage, once per face (face j lies between slots j and j+1); a cell then sums its
            // two faces' corrections over the stages in stage order
            {
                const int nfaces = COWN + 1;  // faces of the own cells
                const int nitems = nfaces * P.nslot;
                for (int k = threadIdx.x; k < nitems; k += blockDim.x) {
                    const int j = k % nfaces, q = k / nfaces;
                    const int rl = c0 - 1 + j, rr = rl + 1;  // unwrapped indices of the two cells
                    const bool el = periodic || (rl >= 0 && rl < P.ncell);
                    const bool er = periodic || (rr >= 0 && rr < P.ncell);
                    // interior sides: the trace, its flux and its spectral radius as the
                    // traced stage's G evaluation computed them; exterior sides from the
                    // boundary condition
                    double uL[M], uR[M], fL[M], fR[M], sL, sR;
                    if (el && er) {
#pragma unroll
                        for (int c = 0; c < M; ++c) {
                            uL[c] = sTr[q][j][1][c];
                            uR[c] = sTr[q][j + 1][0][c];
                            fL[c] = sTf[q][j][1][c];
                            fR[c] = sTf[q][j + 1][0][c];
                        }
                        sL = sSp[q][j][1];
                        sR = sSp[q][j + 1][0];
                    } else if (er) {  // the left side of the mesh: exterior state of side 0
                        double ui[M];
#pragma unroll
                        for (int c = 0; c < M; ++c) {
                            ui[c] = uR[c] = sTr[q][j + 1][0][c];
                            fR[c] = sTf[q][j + 1][0][c];
                        }
                        sR = sSp[q][j + 1][0];
                        exterior_state<PHYS, 1>(P, 0, ui, sAv[q][j + 1], uL);
                        sL = flux_speed_dir<PHYS, 1>(P, uL, 0, fL);
                    } else if (el) {  // the right side: exterior state of side 1
                        double ui[M];
#pragma unroll
                        for (int c = 0; c < M; ++c) {
                            ui[c] = uL[c] = sTr[q][j][1][c];
                            fL[c] = sTf[q][j][1][c];
                        }
                        sL = sSp[q][j][1];
                        exterior_state<PHYS, 1>(P, 1, ui, sAv[q][j], uR);
                        sR = flux_speed_dir<PHYS, 1>(P, uR, 0, fR);
                    } else {
                        continue;  // a face beyond the mesh: no own cell uses it
                    }
                    double alpha = fmax_nonneg(sL, sR);
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        double fhat = 0.5 * (fL[c] + fR[c]) - 0.5 * alpha * (uR[c] - uL[c]);
                        sFc[q][j][0][c] = fhat - fL[c];  // the left cell's right face
                        sFc[q][j][1][c] = fhat - fR[c];  // the right cell's left face
                    }
                }
            }
            __syncthreads();
            double u[M];
            if (own) {
                double dl[M], dr[M];
#pragma unroll
                for (int c = 0; c < M; ++c) dl[c] = dr[c] = 0.0;
                for (int i = 0; i < P.s; ++i) {
                    const int q = P.slot[i];
                    if (q < 0) continue;
#pragma unroll
                    for (int c = 0; c < M; ++c) {
                        dl[c] = fma(P.b[i], sFc[q][lc - 1][1][c], dl[c]);
                        dr[c] = fma(P.b[i], sFc[q][lc][0][c], dr[c]);
                    }
                }
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    double corr = -T.liftp[a] * dr[c] + T.liftm[a] * dl[c];
                    u[c] = fma(dt, P.rhx * corr, acc[c]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < M; ++c) u[c] = acc[c];
            }
            double pts[C::PPT][M];
            limit_block(P, B, S, lc, node, own, u, pts, true, true);
            double amax = 0.0;
#pragma unroll
            for (int j = 0; j < C::PPT; ++j) {
                int p = node + j * NN;
                if (p < C::NSK && own) amax = fmax_nonneg(amax, sk_rate<PHYS, 1>(P, pts[j]));
            }
            unsigned long long abits = dbits(amax);  // non-negative: the bits order as the values
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) abits = umax64(abits, __shfl_xor_sync(0xffffffffu, abits, o));
            if ((threadIdx.x & 31) == 0 && abits > 0ull) atomicMax(B.a0, abits);
            if (own) store_node<1, N, PHYS>(P, unew, gc, node, true, u);
            __syncthreads();
        }
        SlotRead rd;
        if (!grid_barrier(R, (unsigned)(it + 1) * (gridDim.x + (unsigned)R->extra_arrivals), SL, rd)) {
            status = RUN_TIMEOUT;
            break;
        }
        const int fl = rd.flag;
        if (blockIdx.x == 0 && threadIdx.x == 0) {  // the slot used two attempts ahead
            RunSlot *Z = &R->slot[(it + 2) % 3];
            Z->flag = 0;
            Z->nlim = 0ull;
            Z->thmin = dbits(1.0);
            Z->rate = 0ull;
        }
        ++it;
        if (fl == 0) {
            const double rate = bitsd(rd.rate);
            nlim_total += rd.nlim;
            t += dt;
            if (t_end - t <= 1e-14 * fabs(t_end)) t = t_end;
            ++steps;
            restarts += halv;
            halv = 0;
            cur ^= 1;
            rate_last = rate;
            // adaptive: the trial step of the new state; fixed (cfl <= 0): dt0 every step
            dt_try = fmin(cfl > 0.0 ? (rate > 0.0 ? cfl / rate : INFINITY) : R->dt0, t_end - t);
        } else {
            if (++halv > maxh) {
                status = RUN_BOUNDS;
                break;
            }
            dt_try = 0.5 * dt;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        R->t_out = t;
        R->rate_out = rate_last;
        R->steps = steps;
        R->restarts = restarts;
        R->cur_out = cur;
        R->status = status;
        R->nlim_total = nlim_total;
    }
}

template <int N, int PHYS>
cudaError_t run1d_launch(cudaStream_t st, const Params &P, double *u0, double *u1, RunCtl *R, int chunk,
                         int *nblocks) {
    constexpr int NCB = 32;
    using C = RunCfg1D<N, PHYS, NCB>;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_run1d<N, PHYS, NCB>, C::NT, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // chunks of NCB - 2 own cells by default: smaller chunks put more blocks on the GPU but
    // recompute more halo cells and add arrivals at the grid barrier, which costs more than
    // it gains (4096 cells: 26.0 us per step at 30 cells, 26.4 at 27, 30.0 at 20, 47.7 at 7)
    const int slots = nsm * per_sm;
    int cown = chunk > 0 ? chunk : NCB - 2;
    if (cown > NCB - 2) cown = NCB - 2;
    if (cown < 1) cown = 1;
    int nchunks = (P.ncell + cown - 1) / cown;
    int grid = nchunks < slots ? nchunks : slots;
    *nblocks = grid;
    Params Pc = P;
    void *args[] = {&Pc, &u0, &u1, &R, &cown};
    return cudaLaunchCooperativeKernel((void *)k_run1d<N, PHYS, NCB>, dim3(grid), dim3(C::NT), args, 0, st);
}

}  // namespace crkdg
