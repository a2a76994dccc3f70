// dg_ensemble.cuh -- ensembles of 2D Euler problems of uneven size in persistent
// launches.
//
// Every problem keeps its own descriptor (EnsProblem: parameters, buffers, time,
// trial step, restart state).  A persistent kernel of one degree pulls work items
// (problem, first block, block count) from a device counter; for each item whose
// problem takes part in the current attempt it stages the problem's parameters in
// shared memory (only when the problem changes between consecutive items) and runs
// the same block body as the single-problem kernels, so each problem's arithmetic
// is identical to stepping it alone.  Control kernels (one block) open a step
// (trial step of every running problem, clipped to its end time) and close an
// attempt (accept, or halve dt and mark the problem for another attempt, Sec. 4.1).
#pragma once

#include "dg_core.cuh"

namespace crkdg {

template <int N>
__device__ __forceinline__ void ens_bufs(const EnsProblem &E, Bufs &B) {
    B.un = E.u[E.cur];
    B.unew = E.u[E.cur ^ 1];
    B.ustar = E.ustar;
    B.tr = E.tr;
    B.tavg = E.tavg;
    B.flag = &E.sc->flag;
    B.nlim = &E.sc->nlim;
    B.thmin = &E.sc->thmin;
    B.a0 = &E.sc->a0;
    B.aux = E.aux;
    B.ord = E.sc->ord;
    B.tflags = E.tflags;
    B.ntrb = &E.sc->ntrb;
    B.feat = E.feat;
    B.prob = E.prob;
}

template <int N, int KIND>
__device__ __forceinline__ void ens_body(const Params &P, const Bufs &B, int blk) {
    if constexpr (KIND == ENS_INNER) {
        inner_body<2, N, PH_EULER>(P, B, blk);
    } else if constexpr (KIND == ENS_FINAL) {
        final_body<2, N, PH_EULER>(P, B, blk);
    } else if constexpr (KIND == ENS_TROUBLE) {
        trouble_body<2, N, PH_EULER>(P, B, blk);
    } else {
        features_body<2, N, PH_EULER>(P, B, blk);
    }
}

template <int N, int KIND>
constexpr int ens_threads() {
    return KIND == ENS_FEATURES ? 128 : Cfg<2, N, PH_EULER>::NT;
}

// Persistent launch over the work items of one degree.  stage: the troubled-cell
// kernel's ind_stage (ENS_TROUBLE only).
template <int N, int KIND>
__global__ void __launch_bounds__(ens_threads<N, KIND>()) k_ens(EnsProblem *E, const EnsItem *items, int nitems,
                                                                EnsCtl *ctl, int counter, int stage) {
    __shared__ Params sP;
    __shared__ Bufs sB;
    __shared__ int s_item, s_prob;
    if (threadIdx.x == 0) s_prob = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&ctl->counter[counter], 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const EnsItem W = items[it];
        const EnsProblem &pr = E[W.prob];
        if (pr.pending) {  // the same value for every thread of the block
            if (W.prob != s_prob) {
                const int *src = reinterpret_cast<const int *>(&pr.P);
                int *dst = reinterpret_cast<int *>(&sP);
                for (int i = threadIdx.x; i < (int)(sizeof(Params) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
                if (threadIdx.x == 0) ens_bufs<N>(pr, sB);
                __syncthreads();
                if (threadIdx.x == 0) {
                    sP.mode = MODE_STEP;
                    sP.ind_stage = stage;
                    s_prob = W.prob;
                }
                __syncthreads();
            }
            for (int b = 0; b < W.nblk; ++b) {
                ens_body<N, KIND>(sP, sB, W.blk + b);
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void ens_reset_scal(EnsScal *sc) {
    sc->flag = 0;
    sc->nlim = 0ull;
    sc->thmin = dbits(1.0);
    sc->a0 = 0ull;
    sc->ord[0] = sc->ord[1] = ~0ull;
    sc->ntrb = 0ull;
}

// Opens a step: every running problem (of class sel, or all for sel < 0) takes
// its trial step cfl / a0 clipped to its end time.  One block.
__global__ void k_ens_begin(EnsProblem *E, int np, EnsCtl *ctl, int sel) {
    if (threadIdx.x < ENS_COUNTERS) ctl->counter[threadIdx.x] = 0u;
    if (threadIdx.x == 0) ctl->any_pending = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        EnsProblem &p = E[i];
        const bool run = !p.done && p.status == 0 && (sel < 0 || p.klass == sel);
        p.pending = run ? 1 : 0;
        if (!run) continue;
        p.restarts = 0;
        double dt = p.a0 > 0.0 ? p.cfl / p.a0 : INFINITY;
        const double rem = p.t_end - p.t;
        if (dt > rem) dt = rem;
        p.P.dt = dt;
        ens_reset_scal(p.sc);
    }
}

// Clears the work counters before another attempt.  One block.
__global__ void k_ens_reset(EnsCtl *ctl) {
    if (threadIdx.x < ENS_COUNTERS) ctl->counter[threadIdx.x] = 0u;
    if (threadIdx.x == 0) ctl->any_pending = 0;
}

// Closes an attempt: a problem whose stage averages stayed in B^eps accepts the
// step (swaps its states, advances its time, keeps the new rate for the next
// trial step); any other halves dt and stays pending, or stops with
// CRKDG_E_BOUNDS after max_halvings halvings.  One block.
__global__ void k_ens_end(EnsProblem *E, int np, EnsCtl *ctl, int max_halvings) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    if (threadIdx.x < ENS_COUNTERS) ctl->counter[threadIdx.x] = 0u;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        EnsProblem &p = E[i];
        if (!p.pending) continue;
        EnsScal *sc = p.sc;
        if (sc->flag) {
            if (p.restarts >= max_halvings) {
                p.status = 4;  // CRKDG_E_BOUNDS; the state stays at u^n
                p.pending = 0;
                continue;
            }
            p.restarts += 1;
            p.P.dt *= 0.5;
            ens_reset_scal(sc);
            atomicOr(&any, 1);
        } else {
            p.cur ^= 1;
            p.t += p.P.dt;
            p.steps += 1;
            p.restarts_total += p.restarts;
            p.a0 = bitsd(sc->a0);
            p.last_dt = p.P.dt;
            p.last_thmin = bitsd(sc->thmin);
            p.last_nlim = (long long)sc->nlim;
            p.last_ntrb = (long long)sc->ntrb;
            p.last_restarts = p.restarts;
            p.pending = 0;
            if (!(p.t < p.t_end)) p.done = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) ctl->any_pending = any;
}

template <int N, int KIND>
cudaError_t ens_launch_one(int grid, cudaStream_t st, EnsProblem *E, const EnsItem *items, int nitems, EnsCtl *ctl,
                           int counter, int stage) {
    k_ens<N, KIND><<<grid, ens_threads<N, KIND>(), 0, st>>>(E, items, nitems, ctl, counter, stage);
    return cudaGetLastError();
}

template <int N, int KIND>
int ens_occupancy() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ens<N, KIND>, ens_threads<N, KIND>(), 0) != cudaSuccess)
        return 0;
    return b;
}

}  // namespace crkdg
