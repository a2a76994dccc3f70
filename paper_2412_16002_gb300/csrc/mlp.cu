// mlp.cu -- troubled-cell classifier: 44 -> 64 -> 64 -> 1, ReLU, sigmoid, FP32.
//
// Inference (k_mlp_forward_tc): the two hidden layers are dense contractions over
// 128-cell tiles, run on the fifth-generation tensor cores (tcgen05.mma,
// kind::tf32, M = 128, N = 64) with FP32 accumulators in tensor memory.  FP32
// accuracy is kept by the three-product split (3xTF32): every operand x is
// x_hi + x_lo with x_hi = tf32(x) and x_lo = tf32(x - x_hi), and the layer is
// A_hi B_hi + A_hi B_lo + A_lo B_hi.  Bias, ReLU, the 64 -> 1 output layer and
// the sigmoid run on the CUDA cores.  Training (k_mlp_grad): each block takes 64
// samples, runs the forward and backward passes with the activations in shared
// memory, and forms its part of the weight gradients as small contractions over
// its samples before one atomic add per weight; k_mlp_adam applies the Adam
// update.  The loss is the mean binary cross-entropy, written from the logits.
//
// Parameter vector (7105 floats): W1[64][44], b1[64], W2[64][64], b2[64],
// w3[64], b3.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/crkdg.h"

namespace {

constexpr int NIN = CRKDG_MLP_NIN, NH = CRKDG_MLP_NH;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH, NP = OB3 + 1;
static_assert(NP == CRKDG_MLP_NPARAM, "parameter layout");

__device__ __forceinline__ float softplus(float z) { return fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))); }
__device__ __forceinline__ float sigmoidf_(float z) {
    float e = expf(-fabsf(z));
    return z >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e);
}

// ----------------------------------------------------------------------------- tensor-core forward

constexpr int TM = 128;        // cells per tile (MMA M, one TMEM lane per cell)
constexpr int K1 = 48;         // layer-1 K: 44 inputs padded to a multiple of 8
constexpr int TMEM_COLS = 128; // two 64-column FP32 accumulators

// Operand tiles in shared memory, K-major without swizzle: 8-row x 16-byte core
// matrices, core matrix (kc, rg) at ((kc * R/8) + rg) * 128 bytes, so the byte
// offset between core matrices adjacent in K (leading) is R/8 * 128 and between
// row groups (stride) 128.  One MMA (K = 8 TF32) reads two core-matrix columns.
__host__ __device__ constexpr int tile_bytes(int rows, int k) { return rows * k * 4; }
constexpr int SZ_X = tile_bytes(TM, K1), SZ_H = tile_bytes(TM, NH), SZ_W1 = tile_bytes(NH, K1),
              SZ_W2 = tile_bytes(NH, NH);
constexpr int OFF_XH = 0, OFF_XL = OFF_XH + SZ_X, OFF_HH = OFF_XL + SZ_X, OFF_HL = OFF_HH + SZ_H,
              OFF_W1H = OFF_HL + SZ_H, OFF_W1L = OFF_W1H + SZ_W1, OFF_W2H = OFF_W1L + SZ_W1,
              OFF_W2L = OFF_W2H + SZ_W2, OFF_XS = OFF_W2L + SZ_W2,
              SZ_XS = TM * NIN * 4, SMEM_TC = OFF_XS + SZ_XS;  // 194560 bytes
// OFF_XS: the raw features of the next tile (row-major, NIN floats a row), written by
// one bulk asynchronous copy (the tensor memory accelerator's non-tensor form) per tile
static_assert(OFF_XS % 16 == 0 && (NIN * 4) % 16 == 0, "bulk copies move 16-byte multiples");

__device__ __forceinline__ int core_off(int row, int k, int rows) {
    return (((k >> 2) * (rows >> 3) + (row >> 3)) << 7) + ((row & 7) << 4) + ((k & 3) << 2);
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// x rounded to TF32, to nearest with ties away from zero (the rounding of cvt.rna.tf32.f32 for
// every finite or infinite x): half a TF32 unit added to the magnitude bits, 13 low bits cleared
__device__ __forceinline__ float tf32_rna(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
// x -> (hi, lo) for the three-product split
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - hi);
}
// shared-memory matrix descriptor: start, leading and stride byte offsets (>> 4),
// the fixed constant 0b001 at bits 46-48, no swizzle, base offset 0
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9,
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NH >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(da), "l"(db), "r"(IDESC), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// global memory to this CTA's shared memory, completing on mbarrier `bar` (which
// expects the bytes first).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Set when a wait for the tensor cores ran out (1 s); read and cleared by crkdg_mlp_fault.
__device__ unsigned int g_mlp_fault;

// Bounded wait (1 s) for the phase `parity` of an mbarrier (the MMAs of a tile, or a
// tile's bulk copy): true when it completed.
__device__ __forceinline__ bool wait_mma(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(mbar, parity))
        if (globaltimer() - t0 > 1000000000ull) return false;
    return true;
}

// This thread's feature row from the staged tile (zeros past the last row): 16-byte
// reads; eight consecutive rows 176 bytes apart fall on distinct banks.
__device__ __forceinline__ void stage_row(const unsigned char *stage, int rows, int t, float *x) {
    if (t < rows) {
        const float4 *src = reinterpret_cast<const float4 *>(stage) + (size_t)t * (NIN / 4);
#pragma unroll
        for (int q = 0; q < NIN / 4; ++q) {
            float4 v = src[q];
            x[4 * q] = v.x;
            x[4 * q + 1] = v.y;
            x[4 * q + 2] = v.z;
            x[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NIN; ++k) x[k] = 0.0f;
    }
}

// Persistent: each CTA (128 threads, one per cell of a tile) walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; one thread issues the bulk copy of the
// next tile's features into the staging buffer while the current tile's MMAs run,
// and every thread reads its row from there once the copy's mbarrier completes.
__global__ void __launch_bounds__(TM, 1) k_mlp_forward_tc(const float *__restrict__ theta,
                                                          const float *__restrict__ X, int n,
                                                          float *__restrict__ prob) {
    extern __shared__ __align__(1024) unsigned char smt[];
    __shared__ float sb1[NH], sb2[NH], sw3[NH];
    __shared__ __align__(8) unsigned long long s_mbar, s_mbar2, s_xbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fault;
    const int t = threadIdx.x, warp = t >> 5;

    // weights, split, into the B tiles (rows = output units, K = inputs)
    for (int e = t; e < NH * K1; e += TM) {
        const int j = e / K1, k = e - j * K1;
        float hi = 0.0f, lo = 0.0f;
        if (k < NIN) split_tf32(theta[OW1 + j * NIN + k], hi, lo);
        *reinterpret_cast<float *>(smt + OFF_W1H + core_off(j, k, NH)) = hi;
        *reinterpret_cast<float *>(smt + OFF_W1L + core_off(j, k, NH)) = lo;
    }
    for (int e = t; e < NH * NH; e += TM) {
        const int j = e / NH, k = e - j * NH;
        float hi, lo;
        split_tf32(theta[OW2 + e], hi, lo);
        *reinterpret_cast<float *>(smt + OFF_W2H + core_off(j, k, NH)) = hi;
        *reinterpret_cast<float *>(smt + OFF_W2L + core_off(j, k, NH)) = lo;
    }
    if (t < NH) {
        sb1[t] = theta[OB1 + t];
        sb2[t] = theta[OB2 + t];
        sw3[t] = theta[OW3 + t];
    }
    const float b3 = theta[OB3];
    const uint32_t mbar = smem_addr(&s_mbar), mbar2 = smem_addr(&s_mbar2), xbar = smem_addr(&s_xbar);
    const uint32_t a_stage = smem_addr(smt + OFF_XS);
    const int ntiles = (n + TM - 1) / TM;
    auto tile_rows = [&](int tl) { return n - tl * TM < TM ? n - tl * TM : TM; };
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar2) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(xbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fault = 0;
        // the first tile's features (X is 16-byte aligned and rows are 176 bytes)
        if ((int)blockIdx.x < ntiles)
            bulk_load(a_stage, X + (size_t)blockIdx.x * TM * NIN, (uint32_t)(tile_rows(blockIdx.x) * NIN * 4), xbar);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t a_x[2] = {smem_addr(smt + OFF_XH), smem_addr(smt + OFF_XL)};
    const uint32_t a_h[2] = {smem_addr(smt + OFF_HH), smem_addr(smt + OFF_HL)};
    const uint32_t a_w1[2] = {smem_addr(smt + OFF_W1H), smem_addr(smt + OFF_W1L)};
    const uint32_t a_w2[2] = {smem_addr(smt + OFF_W2H), smem_addr(smt + OFF_W2L)};
    constexpr uint32_t LBO_A = (TM / 8) * 128, LBO_B = (NH / 8) * 128, SBO = 128;
    uint32_t phase1 = 0, phase2 = 0, xphase = 0;
    bool inflight = (int)blockIdx.x < ntiles;  // a bulk copy this thread has not seen complete

    // Software pipeline over the CTA's tiles: the next tile's layer-1 MMAs are issued right
    // after this tile's layer-2 MMAs, so they run while the threads wait for layer 2 and
    // form this tile's outputs.  Layer 1 accumulates in columns [0, NH), layer 2 in
    // [NH, 2 NH); mbar (layer 1) and s_mbar2 (layer 2) complete each tile's groups.
    float x[NIN];
    // stage tile `tl`'s features (staged by the bulk copy) into the layer-1 A tile and issue
    // its MMAs, then the copy of the tile after it; false if the copy's wait ran out
    auto start_tile = [&](int tl) -> bool {
        const bool okx = wait_mma(xbar, xphase);
        if (okx) {  // otherwise the copy may still land: drained below at the same phase
            xphase ^= 1u;
            inflight = false;
        }
        if (__syncthreads_or(!okx)) return false;
        stage_row(smt + OFF_XS, tile_rows(tl), t, x);
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            float hi = 0.0f, lo = 0.0f;
            if (k < NIN) split_tf32(x[k], hi, lo);
            *reinterpret_cast<float *>(smt + OFF_XH + core_off(t, k, TM)) = hi;
            *reinterpret_cast<float *>(smt + OFF_XL + core_off(t, k, TM)) = lo;
        }
        proxy_fence();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
        if (t == 0) {
#pragma unroll
            for (int s = 0; s < K1 / 8; ++s) {
                const uint32_t oa = 2 * s * LBO_A, ob = 2 * s * LBO_B;
                mma_tf32(tmem, smem_desc(a_x[0] + oa, LBO_A, SBO), smem_desc(a_w1[0] + ob, LBO_B, SBO), s > 0);
                mma_tf32(tmem, smem_desc(a_x[0] + oa, LBO_A, SBO), smem_desc(a_w1[1] + ob, LBO_B, SBO), 1);
                mma_tf32(tmem, smem_desc(a_x[1] + oa, LBO_A, SBO), smem_desc(a_w1[0] + ob, LBO_B, SBO), 1);
            }
            mma_commit(mbar);
        }
        // the copy of the tile after it (every thread has read the staging buffer and fenced
        // the async proxy before the barrier above)
        const int nxt = tl + gridDim.x;
        if (nxt < ntiles) {
            if (t == 0) bulk_load(a_stage, X + (size_t)nxt * TM * NIN, (uint32_t)(tile_rows(nxt) * NIN * 4), xbar);
            inflight = true;
        }
        return true;
    };

    bool go = (int)blockIdx.x < ntiles;
    if (go && !start_tile(blockIdx.x)) {
        if (t == 0) s_fault = 1;
        go = false;
    }
    for (int tile = blockIdx.x; go && tile < ntiles; tile += gridDim.x) {
        const int r = tile * TM + t;
        bool ok = wait_mma(mbar, phase1);
        phase1 ^= 1u;
        tc_after_sync();
        // layer 1 epilogue: bias, ReLU, split into the layer-2 A tile
        if (ok) {
#pragma unroll
            for (int c = 0; c < NH; c += 16) {
                float v[16];
                tmem_ld16(tmem + lane_base + c, v);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float h = fmaxf(v[i] + sb1[c + i], 0.0f), hi, lo;
                    split_tf32(h, hi, lo);
                    *reinterpret_cast<float *>(smt + OFF_HH + core_off(t, c + i, TM)) = hi;
                    *reinterpret_cast<float *>(smt + OFF_HL + core_off(t, c + i, TM)) = lo;
                }
            }
        }
        proxy_fence();
        tc_before_sync();
        if (__syncthreads_or(!ok)) {
            if (t == 0) s_fault = 1;
            break;
        }
        tc_after_sync();
        if (t == 0) {
#pragma unroll
            for (int s = 0; s < NH / 8; ++s) {
                const uint32_t oa = 2 * s * LBO_A, ob = 2 * s * LBO_B;
                mma_tf32(tmem + NH, smem_desc(a_h[0] + oa, LBO_A, SBO), smem_desc(a_w2[0] + ob, LBO_B, SBO), s > 0);
                mma_tf32(tmem + NH, smem_desc(a_h[0] + oa, LBO_A, SBO), smem_desc(a_w2[1] + ob, LBO_B, SBO), 1);
                mma_tf32(tmem + NH, smem_desc(a_h[1] + oa, LBO_A, SBO), smem_desc(a_w2[0] + ob, LBO_B, SBO), 1);
            }
            mma_commit(mbar2);
        }
        // the next tile's layer 1 while layer 2 of this one runs (its A tile is free: this
        // tile's layer-1 MMAs completed above)
        const int nxt = tile + gridDim.x;
        if (nxt < ntiles && !start_tile(nxt)) {
            if (t == 0) s_fault = 1;
            break;
        }
        ok = wait_mma(mbar2, phase2);
        phase2 ^= 1u;
        tc_after_sync();
        // layer 2 epilogue and the output unit
        float z = b3;
        if (ok) {
#pragma unroll
            for (int c = 0; c < NH; c += 16) {
                float v[16];
                tmem_ld16(tmem + lane_base + NH + c, v);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) z = fmaf(sw3[c + i], fmaxf(v[i] + sb2[c + i], 0.0f), z);
            }
        }
        if (r < n) prob[r] = ok ? sigmoidf_(z) : __int_as_float(0x7fc00000);
        tc_before_sync();
        if (__syncthreads_or(!ok)) {
            if (t == 0) s_fault = 1;
            break;
        }
        tc_after_sync();
    }
    // no copy may still be writing shared memory when the CTA exits
    if (inflight && !wait_mma(xbar, xphase)) s_fault = 1;
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (t == 0 && s_fault) atomicOr(&g_mlp_fault, 1u);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

constexpr int SB = 64;  // samples per block in the gradient kernel

__global__ void __launch_bounds__(SB) k_mlp_grad(const float *__restrict__ theta, const float *__restrict__ X,
                                                 const float *__restrict__ y, int n, float inv_total,
                                                 float *__restrict__ grad, float *__restrict__ loss) {
    extern __shared__ float sm[];
    float *w = sm;                  // NP
    float *sx = w + NP;             // SB x NIN
    float *sh1 = sx + SB * NIN;     // SB x NH  (h1)
    float *sd1 = sh1 + SB * NH;     // SB x NH  (d a1)
    float *sd2 = sd1 + SB * NH;     // SB x NH  (d a2)
    float *sdz = sd2 + SB * NH;     // SB
    float *sh2 = sdz + SB;          // SB x NH  (h2)
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = theta[i];
    const int t = threadIdx.x;
    const int r = blockIdx.x * SB + t;
    const bool valid = r < n;
    for (int k = 0; k < NIN; ++k) sx[t * NIN + k] = valid ? X[(size_t)r * NIN + k] : 0.0f;
    __syncthreads();
    // forward, one sample per thread
    float a1[NH];
    for (int j = 0; j < NH; ++j) {
        float a = w[OB1 + j];
        for (int k = 0; k < NIN; ++k) a = fmaf(w[OW1 + j * NIN + k], sx[t * NIN + k], a);
        a1[j] = a;
        sh1[t * NH + j] = fmaxf(a, 0.0f);
    }
    float z = w[OB3];
    for (int j = 0; j < NH; ++j) {
        float a = w[OB2 + j];
        for (int i = 0; i < NH; ++i) a = fmaf(w[OW2 + j * NH + i], sh1[t * NH + i], a);
        float h = fmaxf(a, 0.0f);
        sh2[t * NH + j] = h;
        sd2[t * NH + j] = a > 0.0f ? 1.0f : 0.0f;  // ReLU mask, scaled below
        z = fmaf(w[OW3 + j], h, z);
    }
    float yy = valid ? y[r] : 0.0f;
    float dz = valid ? (sigmoidf_(z) - yy) * inv_total : 0.0f;
    if (valid) atomicAdd(loss, (softplus(z) - yy * z) * inv_total);
    sdz[t] = dz;
    // backward through the layers of this sample
    for (int j = 0; j < NH; ++j) sd2[t * NH + j] *= dz * w[OW3 + j];
    for (int i = 0; i < NH; ++i) {
        float s = 0.0f;
        for (int j = 0; j < NH; ++j) s = fmaf(sd2[t * NH + j], w[OW2 + j * NH + i], s);
        sd1[t * NH + i] = a1[i] > 0.0f ? s : 0.0f;
    }
    __syncthreads();
    // weight gradients: contractions over the block's samples, one atomic per weight
    for (int e = t; e < NH * NIN; e += SB) {
        int j = e / NIN, k = e - j * NIN;
        float s = 0.0f;
        for (int q = 0; q < SB; ++q) s = fmaf(sd1[q * NH + j], sx[q * NIN + k], s);
        atomicAdd(&grad[OW1 + e], s);
    }
    for (int e = t; e < NH * NH; e += SB) {
        int j = e / NH, i = e - j * NH;
        float s = 0.0f;
        for (int q = 0; q < SB; ++q) s = fmaf(sd2[q * NH + j], sh1[q * NH + i], s);
        atomicAdd(&grad[OW2 + e], s);
    }
    if (t < NH) {
        float s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        for (int q = 0; q < SB; ++q) {
            s1 += sd1[q * NH + t];
            s2 += sd2[q * NH + t];
            s3 = fmaf(sdz[q], sh2[q * NH + t], s3);
        }
        atomicAdd(&grad[OB1 + t], s1);
        atomicAdd(&grad[OB2 + t], s2);
        atomicAdd(&grad[OW3 + t], s3);
    }
    if (t == 0) {
        float s = 0.0f;
        for (int q = 0; q < SB; ++q) s += sdz[q];
        atomicAdd(&grad[OB3], s);
    }
}

__global__ void k_mlp_adam(float *theta, float *m, float *v, const float *grad, float lr, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float g = grad[i];
    float mi = b1 * m[i] + (1.0f - b1) * g;
    float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

size_t grad_smem() { return sizeof(float) * (NP + SB * NIN + 4 * SB * NH + SB); }

}  // namespace

extern "C" {

crkdg_status crkdg_mlp_forward(const float *params, const float *X, int n, float *prob, void *stream) {
    if (!params || !X || !prob || n < 0) return CRKDG_E_ARG;
    if (n == 0) return CRKDG_OK;
    if (((uintptr_t)X & 15u) != 0) return CRKDG_E_ARG;  // rows are read as 16-byte vectors
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CRKDG_E_CUDA;
    static int configured_dev = -1;  // the attribute is per device
    if (configured_dev != dev) {
        if (cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC) !=
            cudaSuccess)
            return CRKDG_E_CUDA;
        configured_dev = dev;
    }
    const int ntiles = (n + TM - 1) / TM;
    const int grid = ntiles < nsm ? ntiles : nsm;  // one CTA per SM (190 KB of shared memory each)
    k_mlp_forward_tc<<<grid, TM, SMEM_TC, (cudaStream_t)stream>>>(params, X, n, prob);
    return cudaGetLastError() == cudaSuccess ? CRKDG_OK : CRKDG_E_CUDA;
}

crkdg_status crkdg_mlp_fault(int *fault) {
    if (!fault) return CRKDG_E_ARG;
    unsigned int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_mlp_fault, sizeof(v)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_mlp_fault, &zero, sizeof(zero)) != cudaSuccess)
        return CRKDG_E_CUDA;
    *fault = (int)v;
    return CRKDG_OK;
}

crkdg_status crkdg_mlp_grad(const float *params, const float *X, const float *y, int n, float *grad, float *loss,
                            void *stream) {
    if (!params || !X || !y || !grad || !loss || n <= 0) return CRKDG_E_ARG;
    static bool configured = false;
    if (!configured) {
        if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()) !=
            cudaSuccess)
            return CRKDG_E_CUDA;
        configured = true;
    }
    k_mlp_grad<<<(n + SB - 1) / SB, SB, grad_smem(), (cudaStream_t)stream>>>(params, X, y, n, 1.0f / (float)n, grad,
                                                                            loss);
    return cudaGetLastError() == cudaSuccess ? CRKDG_OK : CRKDG_E_CUDA;
}

crkdg_status crkdg_mlp_adam(float *params, float *m, float *v, const float *grad, int step, float lr, void *stream) {
    if (!params || !m || !v || !grad || step < 1 || !(lr > 0.0f)) return CRKDG_E_ARG;
    float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
    k_mlp_adam<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, lr, c1, c2);
    return cudaGetLastError() == cudaSuccess ? CRKDG_OK : CRKDG_E_CUDA;
}

}  // extern "C"
