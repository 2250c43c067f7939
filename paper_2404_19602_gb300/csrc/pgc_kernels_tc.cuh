// pgc_kernels_tc.cuh -- the streaming work of one time step (phase 1) for the two-input shape
// (total degree 5: P = 21 coefficients, 6 x 6 tensor Gauss nodes: Q = 36) with the
// reconstruction at the nodes (Eq. (23)) on the fifth-generation tensor cores.
//
// Per 128-particle tile the reconstruction is the contraction
//     K_c[i][q] = sum_h khat_c[i][h] Psi_h(z_q),   c = x, y,
// i.e. D = A B^T with A = [128 particles x 21 coefficients] and B = [36 nodes x 21 coefficients],
// dense, with FP32 accumulation in tensor memory.  FP32 operands are split into FP16 pairs
// a = a_hi + a_lo (a_hi = fp16(a), a_lo = fp16(a - a_hi)), so that with the three products
// A_hi B_hi + A_hi B_lo + A_lo B_hi the node values carry ~22 significant bits, the precision
// class of the FP32 FMA reconstruction (mode PGC_TC_F16X3); mode PGC_TC_F16 takes the single
// product A_hi B_hi (FP16 inputs, ~11 bits).  Operands are scaled by 2^10 each (exact) so that
// the low parts stay in the normal FP16 range; the node values are scaled back by 2^-20.
//
// Everything after the reconstruction -- the drift before it, the flight-time screen, the
// histogram f^{n+1} in the block's shared-memory window, the collider queue, the moments --
// follows phase1_pass of pgc_kernels.cuh, per particle.
//
// One CTA per SM (its shared memory allows no second one), 4 warpgroups of 128 threads; each
// warpgroup owns one tile per iteration: thread t of the warpgroup carries particle t of the
// tile, writes row t of the operands, and reads row t of the accumulators (TMEM lane t).  TMEM:
// 512 columns per CTA, warpgroup g uses [128 g, 128 g + 96): D_x in the first 48, D_y in the
// next 48 (N = 48: 36 nodes padded).  One thread per warpgroup issues the 12 (or 4) MMAs of a
// tile and commits them to the warpgroup's mbarrier; every wait on it is bounded and a wait
// that gives up sets bit 0 of the device error counter.
#pragma once

#include "pgc_kernels.cuh"
#include "pgc_umma.cuh"

namespace pgc {

constexpr int kTcWG = 4;                    // warpgroups per CTA
constexpr int kTcThreads = 128 * kTcWG;
constexpr int kTcK = 32;                    // K padded to two K = 16 MMA steps (21 coefficients)
constexpr int kTcN = 48;                    // N padded (36 nodes)
constexpr int kTcColsWG = 128;              // TMEM columns per warpgroup
constexpr uint32_t kTcCols = kTcColsWG * kTcWG;
constexpr int kTcOpBytes = 128 * kTcK * 2;  // one FP16 operand tile [128 x 32]
constexpr float kTcScale = 1024.0f;         // 2^10 per operand
constexpr float kTcUnscale = 1.0f / (1024.0f * 1024.0f);
constexpr uint32_t kTcWaitTries = 1u << 20;
constexpr float kTcEscape = 32.0f;          // |coefficient| beyond which the tile row is not trusted

// dynamic shared memory: window | A operands [wg][x_hi, x_lo, y_hi, y_lo] | B [hi, lo] | moment
// partials [warps][Q*3] | mbarriers [wg] | TMEM base
template <int Q> struct TcSmem {
    static constexpr size_t win = (size_t)Q * kWinWords * 4;
    static constexpr size_t offA = (win + 1023) / 1024 * 1024;
    static constexpr size_t offB = offA + (size_t)kTcWG * 4 * kTcOpBytes;
    static constexpr size_t offMom = offB + 2 * (size_t)kTcN * kTcK * 2;
    static constexpr size_t offBar = offMom + (size_t)(kTcThreads / 32) * Q * 3 * 8;
    static constexpr size_t bytes = offBar + 8 * kTcWG + 16;
};

__device__ __forceinline__ void wg_bar(int wg) { asm volatile("bar.sync %0, 128;" ::"r"(1 + wg) : "memory"); }

// 16-byte asynchronous global -> shared copy; with ok false nothing is read and zeros land.
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src, bool ok)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst_smem)), "l"(src), "r"(ok ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Prefetch of one tile's coefficients (all 2P planes, 128 particles from i0) into the
// warpgroup's operand area as raw FP32 [2P][128], 16-byte chunks spread over its 128 threads.
// Chunks at or beyond ld (the padded plane length, a multiple of 64) are not read.
template <int P>
__device__ __forceinline__ void prefetch_tile(unsigned char *stage, const float *khat, int64_t ld, int64_t i0, int t)
{
    for (int j = t; j < 2 * P * 32; j += 128) {
        const int h = j >> 5, c = j & 31;
        const int64_t col = i0 + 4 * c;
        const bool ok = col < ld;
        const float *src = khat + (int64_t)h * ld + (ok ? col : 0);
        cp_async16(stage + h * 512 + 16 * c, src, ok);
    }
    cp_async_commit();
}

template <int P, int Q>
__global__ void __launch_bounds__(kTcThreads, 1)
k_phase1_tc(const __grid_constant__ StepArgs<P, Q, float> a, int mode)
{
    static_assert(TensorShape<P, Q>::value, "tensor-core reconstruction is compiled for the 21 x 36 shape");
    using S = TcSmem<Q>;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint32_t *swin = reinterpret_cast<uint32_t *>(smem);
    unsigned char *sA = smem + S::offA;
    unsigned char *sB = smem + S::offB;
    float2 *smom = reinterpret_cast<float2 *>(smem + S::offMom);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + S::offBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + S::offBar + 8 * kTcWG);

    const int tid = threadIdx.x, wg = tid >> 7, t = tid & 127, warp = tid >> 5, lane = tid & 31;
    const Phys<float> &ph = a.ph;
    const Nodes<P, Q, float> &nd = a.nd;
    const int64_t NN = (int64_t)ph.Nk * ph.Nk;
    const int bid = blockIdx.x, nb = gridDim.x;

    // --- set-up: window, moment partials, operands (zero padding), B = scaled Psi split ---
    if (a.use_win)
        for (int j = tid; j < Q * kWinWords; j += kTcThreads) swin[j] = 0u;
    for (int j = tid; j < (kTcThreads / 32) * Q * 3; j += kTcThreads) acc_zero(smom[j]);
    for (int j = tid; j < kTcWG * 4 * kTcOpBytes / 16; j += kTcThreads)
        reinterpret_cast<uint4 *>(sA)[j] = make_uint4(0u, 0u, 0u, 0u);
    for (int j = tid; j < kTcN * kTcK / 2; j += kTcThreads) {
        const int n = j / (kTcK / 2), k = 2 * (j % (kTcK / 2));
        const float b0 = (n < Q && k < P) ? nd.psi[n * P + k] * kTcScale : 0.0f;
        const float b1 = (n < Q && k + 1 < P) ? nd.psi[n * P + k + 1] * kTcScale : 0.0f;
        uint32_t hi, lo;
        split_f16x2(b0, b1, hi, lo);
        *reinterpret_cast<uint32_t *>(sB + umma_off(n, k, kTcK)) = hi;
        *reinterpret_cast<uint32_t *>(sB + kTcN * kTcK * 2 + umma_off(n, k, kTcK)) = lo;
    }
    if (tid == 0) {
        for (int g = 0; g < kTcWG; ++g) mbar_init(&mbar[g], 1);
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, kTcCols);
        tmem_relinquish();
    }
    // housekeeping for the next steps (as phase1_block)
    if (bid == 0 && tid == 0) {
        *a.qcount_next = 0u;
        if (a.tilectr_next) *a.tilectr_next = 0u;
    }
    {
        uint4 *hc = reinterpret_cast<uint4 *>(a.Hclear);
        const int64_t n4 = a.hist_elems >> 2;
        for (int64_t j = (int64_t)bid * kTcThreads + tid; j < n4; j += (int64_t)nb * kTcThreads)
            hc[j] = make_uint4(0u, 0u, 0u, 0u);
        if (bid == 0)
            for (int64_t j = (n4 << 2) + tid; j < a.hist_elems; j += kTcThreads) a.Hclear[j] = 0u;
        if (a.mark_clear) {
            uint4 *mc = reinterpret_cast<uint4 *>(a.mark_clear);
            for (int64_t j = (int64_t)bid * kTcThreads + tid; j < (a.mark_words >> 2); j += (int64_t)nb * kTcThreads)
                mc[j] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot + (uint32_t)(wg * kTcColsWG);
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's TMEM lanes
    const uint32_t idesc = umma_idesc_f16(128, kTcN);
    unsigned char *opA = sA + (size_t)wg * 4 * kTcOpBytes;               // x_hi, x_lo, y_hi, y_lo
    float2 *smw = smom + warp * (Q * 3);

    const int64_t ntiles = (a.N + 127) / 128;
    const int64_t stride = (int64_t)nb * kTcWG;
    const int64_t iters = (ntiles + stride - 1) / stride;
    int64_t since_flush = 0;
    uint32_t parity = 0, wait_tries = kTcWaitTries;
    bool tc_err = false;
    unsigned int oog = 0u;
    const bool out_step = a.out_step != 0, use_win = a.use_win != 0;

    auto tile_base = [&](int64_t it) { return (it * stride + (int64_t)bid * kTcWG + wg) * 128; };
    if (iters > 0) prefetch_tile<P>(opA, a.khat, a.ld, tile_base(0), t);

    for (int64_t it = 0; it < iters; ++it) {
        if (use_win && since_flush + kTcThreads > 65535) {   // CTA-uniform (see phase1_block)
            __syncthreads();
            flush_window<Q>(swin, a.Hnext, ph.Nk, a.win_r0);
            __syncthreads();
            for (int j = tid; j < Q * kWinWords; j += kTcThreads) swin[j] = 0u;
            __syncthreads();
            since_flush = 0;
        }
        since_flush += kTcThreads;
        const int64_t i = tile_base(it) + t;
        const bool valid = i < a.N;

        // this tile's coefficients, prefetched into the operand area; read by every thread
        // before any thread writes its operand rows over them
        cp_async_wait_all();
        wg_bar(wg);
        float raw[2 * P];
        {
            const float *stage = reinterpret_cast<const float *>(opA);
#pragma unroll
            for (int h = 0; h < 2 * P; ++h) raw[h] = valid ? stage[h * 128 + t] : 0.0f;
        }
        wg_bar(wg);
        // the padding core matrix of this row (k = 24..31) held staged data: zero in all four operands
#pragma unroll
        for (int o = 0; o < 4; ++o)
            *reinterpret_cast<uint4 *>(opA + o * kTcOpBytes + umma_off(t, 24, kTcK)) = make_uint4(0u, 0u, 0u, 0u);

        // drift (Eq. (17)) and the operand rows of this particle
        float amax = 0.0f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float v[P];
#pragma unroll
            for (int h = 0; h < P; ++h) v[h] = raw[c * P + h];
            if (c == 0) {
#pragma unroll
                for (int h = 0; h < P; ++h)
                    if (nd.drift_mask & (1u << h)) {
                        v[h] -= valid ? nd.dhat[h] : 0.0f;
                        if (valid) a.khat[(int64_t)h * a.ld + i] = v[h];
                    }
            }
#pragma unroll
            for (int h = 0; h < P; ++h) amax = fmaxf(amax, fabsf(v[h]));
            unsigned char *hiA = opA + (2 * c) * kTcOpBytes, *loA = hiA + kTcOpBytes;
#pragma unroll
            for (int kc = 0; kc < 3; ++kc) {   // core matrices k = 0..7, 8..15, 16..23 (24..31 stay zero)
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k0 = kc * 8 + 2 * j;
                    const float a0 = (k0 < P) ? v[k0] * kTcScale : 0.0f;
                    const float a1 = (k0 + 1 < P) ? v[k0 + 1] * kTcScale : 0.0f;
                    split_f16x2(a0, a1, hw[j], lw[j]);
                }
                *reinterpret_cast<uint4 *>(hiA + umma_off(t, kc * 8, kTcK)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(loA + umma_off(t, kc * 8, kTcK)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        }
        const bool escape = !(amax < kTcEscape);   // huge or non-finite coefficients: not trusted here

        // the warpgroup's operands are complete: one thread issues the MMAs
        fence_async_smem();
        tc_fence_before();
        wg_bar(wg);
        if (t == 0) {
            tc_fence_after();
            const uint32_t bhi = smem_u32(sB), blo = bhi + kTcN * kTcK * 2;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const uint32_t d = tmem + (uint32_t)(c * kTcN);
                const uint32_t ahi = smem_u32(opA + (2 * c) * kTcOpBytes), alo = ahi + kTcOpBytes;
#pragma unroll
                for (int ks = 0; ks < kTcK / 16; ++ks) {
                    const uint32_t o = (uint32_t)ks * 2 * kUmmaLBO;
                    const uint32_t sbo = umma_sbo(kTcK);
                    umma_f16_ss(d, umma_sdesc(ahi + o, kUmmaLBO, sbo), umma_sdesc(bhi + o, kUmmaLBO, sbo), idesc, ks > 0);
                    if (mode == 1) {
                        umma_f16_ss(d, umma_sdesc(ahi + o, kUmmaLBO, sbo), umma_sdesc(blo + o, kUmmaLBO, sbo), idesc, true);
                        umma_f16_ss(d, umma_sdesc(alo + o, kUmmaLBO, sbo), umma_sdesc(bhi + o, kUmmaLBO, sbo), idesc, true);
                    }
                }
            }
            umma_commit(&mbar[wg]);
        }
        if (!mbar_wait_bounded(&mbar[wg], parity, wait_tries)) {
            tc_err = true;
            wait_tries = 1;   // the kernel runs to its end quickly; the host reports the error
        }
        parity ^= 1u;
        tc_fence_after();
        // the operands are consumed: the next tile's coefficients stream in behind this tile's work
        if (it + 1 < iters && !tc_err) prefetch_tile<P>(opA, a.khat, a.ld, tile_base(it + 1), t);

        // pass 1: |k|^2 at the nodes, the bound of the majorant
        float kkmax_s = 0.0f;
#pragma unroll
        for (int c0 = 0; c0 < Q; c0 += 8) {
            float vx[8], vy[8];
            if (c0 + 8 <= Q) {
                tmem_ld8(trow + c0, vx);
                tmem_ld8(trow + kTcN + c0, vy);
            } else {
                tmem_ld4(trow + c0, vx);
                tmem_ld4(trow + kTcN + c0, vy);
            }
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (c0 + j < Q) kkmax_s = fmaxf(kkmax_s, fmaf(vx[j], vx[j], vy[j] * vy[j]));
        }
        const float kkmax = kkmax_s * (kTcUnscale * kTcUnscale);
        const U4 rr = philox4x32_10((uint32_t)i, a.stream_id, a.step, 0u, a.key0, a.key1);
        const bool maybe = valid && (escape || screen_maybe(ph, nd, kkmax, rr.x));
        const bool fin = valid && !maybe;

        // pass 2: cells of the finished particles into f^{n+1}, and their moments (node q,
        // quantity j is value 3 q + j of a stream of warp reduce-scatters, 16 values each)
        if (__any_sync(0xffffffffu, fin)) {   // warp-uniform: tcgen05.ld is .sync.aligned
            float buf[16];
#pragma unroll
            for (int c0 = 0; c0 < Q; c0 += 8) {
                float vx[8], vy[8];
                if (c0 + 8 <= Q) {
                    tmem_ld8(trow + c0, vx);
                    tmem_ld8(trow + kTcN + c0, vy);
                } else {
                    tmem_ld4(trow + c0, vx);
                    tmem_ld4(trow + kTcN + c0, vy);
                }
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int q = c0 + j;
                    if (q >= Q) continue;
                    const float kx = vx[j] * kTcUnscale, ky = vy[j] * kTcUnscale;
                    if (fin) {
                        int r, l;
                        if (!cell_rl(ph, nd.lkx[q], kx, ky, r, l)) {
                            ++oog;
                        } else {
                            const int rw = r - a.win_r0, lw = l - a.win_r0;
                            if (use_win && (unsigned)rw < (unsigned)kWin && (unsigned)lw < (unsigned)kWin)
                                atomicAdd(&swin[q * kWinWords + rw * (kWin / 2) + (lw >> 1)], 1u << ((lw & 1) << 4));
                            else
                                atomicAdd(&a.Hnext[(int64_t)q * NN + r * ph.Nk + l], 1u);
                        }
                    }
                    if (out_step) {
                        float o[3] = {0.0f, 0.0f, 0.0f};
                        if (fin) observe_fast(ph, kx - nd.xs[q], ky, nd.eps0[q], o[0], o[1], o[2]);
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            const int idx = 3 * q + m;
                            buf[idx & 15] = o[m];
                            if ((idx & 15) == 15 || idx == 3 * Q - 1) {
                                for (int z = (idx & 15) + 1; z < 16; ++z) buf[z] = 0.0f;
                                warp_scatter16_add(buf, smw + (idx & ~15), (idx & 15) + 1, lane);
                            }
                        }
                    }
                }
            }
        }

        // colliders go to the queue (warp-aggregated append)
        const unsigned int mask = __ballot_sync(0xffffffffu, maybe);
        if (mask) {
            const int leader = __ffs(mask) - 1;
            uint32_t basepos = 0;
            if (lane == leader) basepos = atomicAdd(a.qcount, (uint32_t)__popc(mask));
            basepos = __shfl_sync(0xffffffffu, basepos, leader);
            if (maybe) {
                a.queue[basepos + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)i;
                if (a.mark) atomicOr(&a.mark[i >> 5], 1u << (i & 31));
            }
        }
        tc_fence_before();   // TMEM reads of this tile are ordered before the next tile's MMAs
    }

    oog = warp_sum(oog);
    if (lane == 0 && oog) atomicAdd(&a.counters[4], (unsigned long long)oog);
    if (tc_err) atomicOr(&a.counters[6], 1ull);
    __syncthreads();
    if (use_win) flush_window<Q>(swin, a.Hnext, ph.Nk, a.win_r0);
    if (out_step)
        for (int j = tid; j < Q * 3; j += kTcThreads) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kTcThreads / 32; ++w) s += acc_value(smom[w * (Q * 3) + j]);
            a.part1[(int64_t)bid * (Q * 3) + j] = s;
        }
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, kTcCols);
}

}  // namespace pgc
