// Row update (step + gradient + L-BFGS pair) with TMA-staged inputs.
//
// Same arithmetic as k_update<TR, TD, CPL, true, true> without a W term, but
// the read streams (R, C R, D, C D, G and the stored pairs) of a tile of rows
// are brought into shared memory by 1-D bulk copies (cp.async.bulk) tracked by
// an mbarrier transaction count, several tiles ahead of the compute.  Memory
// parallelism then no longer depends on how many warps the registers allow.
// Every wait is bounded: on expiry the kernel raises the device error flag and
// returns (the host turns it into LORADS_ERR_TIMEOUT).
#pragma once

#include "kernels.cuh"

namespace lorads {

constexpr int kTmaStages = 3;
constexpr unsigned kWaitLimit = 1u << 26;      // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false when the limit expired
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Shared-memory footprint of one stage for tiles of `rows` rows.
template <typename TR, typename TD>
__host__ __device__ inline size_t tma_stage_bytes(int rows, int ld) {
    return (size_t)rows * ld * (2 * sizeof(TR) + (3 + 2 * (kMaxMem - 1)) * sizeof(TD));
}

template <typename TR, typename TD, int CPL>
__global__ void __launch_bounds__(kThreads, 1)
k_update_tma(ProbDev p, TR* __restrict__ R, TR* __restrict__ CR, const TD* __restrict__ D,
             const TD* __restrict__ CD, TD* __restrict__ G, TD* __restrict__ hist, int64_t slot_stride, int ld,
             int L, int Q, const double* __restrict__ y, const dfloat* __restrict__ ydf, void* __restrict__ zrow_v,
             Ctrl* ctrl, double* __restrict__ part, const Ctrl* gate, int ph) {
    if (gated_off(gate, ph)) return;
    using AR = arith_t<TR>;
    using AD = arith_t<TD>;
    using PA = part_t<TR, TD>;
    using RS = rowscalar_t<TR, TD>;
    using ZS = zrow_t<TD, TR>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kTmaStages];
    __shared__ int abort_flag;

    ZS* __restrict__ zrow = static_cast<ZS*>(zrow_v);
    const RS rho_r = RS(ctrl->rho);
    const double taud = ctrl->tau;
    const AR tau = AR(taud);
    const AD tau_d = AD(taud);
    const int nold = ctrl->old_count;
    const int ns = ctrl->new_slot;
    TD* Snew = hist + (int64_t)(2 * ns) * slot_stride;
    TD* Ynew = hist + (int64_t)(2 * ns + 1) * slot_stride;
    const TD* So[kMaxMem - 1];
    const TD* Yo[kMaxMem - 1];
#pragma unroll
    for (int t = 0; t < kMaxMem - 1; ++t) {
        const int s = ctrl->old_slots[t < nold ? t : 0];
        So[t] = hist + (int64_t)(2 * s) * slot_stride;
        Yo[t] = hist + (int64_t)(2 * s + 1) * slot_stride;
    }

    const int rows_per_tile = kThreads / L;
    const int64_t ntiles = (p.n + rows_per_tile - 1) / rows_per_tile;
    const size_t rowbR = (size_t)ld * sizeof(TR), rowbD = (size_t)ld * sizeof(TD);
    const size_t stage_bytes = tma_stage_bytes<TR, TD>(rows_per_tile, ld);
    // offsets inside a stage
    const size_t oR = 0, oCR = oR + rows_per_tile * rowbR, oD = oCR + rows_per_tile * rowbR;
    const size_t oCD = oD + rows_per_tile * rowbD, oG = oCD + rows_per_tile * rowbD, oH = oG + rows_per_tile * rowbD;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTmaStages; ++s) mbar_init(&bars[s], 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // producer: one thread issues the copies of the block's j-th tile into stage j % S
    auto issue = [&](int64_t j) {
        const int64_t tile = blockIdx.x + j * (int64_t)gridDim.x;
        if (tile >= ntiles) return;
        const int64_t i0 = tile * rows_per_tile;
        const int rows = (int)((p.n - i0) < rows_per_tile ? (p.n - i0) : rows_per_tile);
        unsigned char* st = smem + (size_t)(j % kTmaStages) * stage_bytes;
        uint64_t* bar = &bars[j % kTmaStages];
        const uint32_t bR = (uint32_t)(rows * rowbR), bD = (uint32_t)(rows * rowbD);
        mbar_expect_tx(bar, 2 * bR + (3 + 2 * nold) * bD);
        bulk_load(st + oR, R + i0 * ld, bR, bar);
        bulk_load(st + oCR, CR + i0 * ld, bR, bar);
        bulk_load(st + oD, D + i0 * ld, bD, bar);
        bulk_load(st + oCD, CD + i0 * ld, bD, bar);
        bulk_load(st + oG, G + i0 * ld, bD, bar);
        for (int t = 0; t < nold; ++t) {
            bulk_load(st + oH + (size_t)(2 * t) * rows_per_tile * rowbD, So[t] + i0 * ld, bD, bar);
            bulk_load(st + oH + (size_t)(2 * t + 1) * rows_per_tile * rowbD, Yo[t] + i0 * ld, bD, bar);
        }
    };
    if (threadIdx.x == 0)
        for (int j = 0; j < kTmaStages; ++j) issue(j);

    PA accq[PU_N];
#pragma unroll
    for (int q = 0; q < PU_N; ++q) accq[q] = PA(0);
    const int lig = threadIdx.x & (L - 1);
    const int rloc = threadIdx.x / L;                 // row of the tile this group handles

    for (int64_t j = 0;; ++j) {
        const int64_t tile = blockIdx.x + j * (int64_t)gridDim.x;
        if (tile >= ntiles) break;
        const int s = (int)(j % kTmaStages);
        const uint32_t parity = (uint32_t)((j / kTmaStages) & 1);
        if (!mbar_wait(&bars[s], parity)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) {
            if (threadIdx.x == 0) ctrl->dev_error = 1;
            return;
        }
        const unsigned char* st = smem + (size_t)s * stage_bytes;
        const int64_t i = tile * rows_per_tile + rloc;
        const bool act = i < p.n;
        const TR* sR = reinterpret_cast<const TR*>(st + oR) + (size_t)rloc * ld + lig * 4;
        const TR* sCR = reinterpret_cast<const TR*>(st + oCR) + (size_t)rloc * ld + lig * 4;
        const TD* sD = reinterpret_cast<const TD*>(st + oD) + (size_t)rloc * ld + lig * 4;
        const TD* sCD = reinterpret_cast<const TD*>(st + oCD) + (size_t)rloc * ld + lig * 4;
        const TD* sG = reinterpret_cast<const TD*>(st + oG) + (size_t)rloc * ld + lig * 4;
        Unit<TR> r[CPL], cr[CPL];
        Unit<TD> d[CPL];
        AR rr = AR(0);
        if (act) {
            Unit<TD> cd[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                if (c * L + lig < Q) {
                    r[c].load(sR + c * L * 4);
                    cr[c].load(sCR + c * L * 4);
                    d[c].load(sD + c * L * 4);
                    cd[c].load(sCD + c * L * 4);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        r[c].v[e] = 0; cr[c].v[e] = 0; d[c].v[e] = 0; cd[c].v[e] = 0;
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    r[c].v[e] = step_add<AR, AD>(AR(r[c].v[e]), tau, tau_d, AD(d[c].v[e]));
                    cr[c].v[e] = step_add<AR, AD>(AR(cr[c].v[e]), tau, tau_d, AD(cd[c].v[e]));
                }
            }
            store_row<TR, CPL>(r, R, i, ld, L, Q, lig);
            store_row<TR, CPL>(cr, CR, i, ld, L, Q, lig);
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) rr = sq_add<AR>(rr, AR(r[c].v[e]));
        }
        AR coef = AR(0);
        if (p.dk != nullptr) {
            rr = group_sum(rr, L);
            if (act) {
                const int k = __ldg(p.dk + i);
                if (k >= 0) {
                    const RS a = ld_scalar<RS>(p.da, p.da_df, i);
                    const RS z = a * RS(rr) - ld_scalar<RS>(p.b, p.b_df, k);
                    const RS yv = ydf ? ld_scalar<RS>(y, ydf, k) : RS(__ldg(y + k));
                    coef = AR(a * (yv - rho_r * z));
                    if (lig == 0) {
                        accq[PU_ZZ] += PA(z * z);
                        if (zrow != nullptr) zrow[i] = ZS(z);
                    }
                }
            }
        }
        if (act) {
            Unit<TD> g[CPL], gold[CPL], sn[CPL], yn[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                if (c * L + lig < Q) gold[c].load(sG + c * L * 4);
                else
#pragma unroll
                    for (int e = 0; e < 4; ++e) gold[c].v[e] = 0;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    g[c].v[e] = grad_elem<AR, AD>(AR(cr[c].v[e]), coef, AR(r[c].v[e]));
                    sn[c].v[e] = tau_d * AD(d[c].v[e]);
                    yn[c].v[e] = AD(g[c].v[e]) - AD(gold[c].v[e]);
                }
            }
            store_row<TD, CPL>(sn, Snew, i, ld, L, Q, lig);
            store_row<TD, CPL>(yn, Ynew, i, ld, L, Q, lig);
            store_row<TD, CPL>(g, G, i, ld, L, Q, lig);
            accq[PU_GYN] += dot_units<AD>(g, yn);
            accq[PU_SYN] += dot_units<AD>(sn, yn);
            accq[PU_YYN] += dot_units<AD>(yn, yn);
            accq[PU_GG] += dot_units<AD>(g, g);
#pragma unroll
            for (int t = 0; t < kMaxMem - 1; ++t) {
                if (t < nold) {
                    const TD* sS = reinterpret_cast<const TD*>(st + oH + (size_t)(2 * t) * rows_per_tile * rowbD) +
                                   (size_t)rloc * ld + lig * 4;
                    const TD* sY = reinterpret_cast<const TD*>(st + oH + (size_t)(2 * t + 1) * rows_per_tile * rowbD) +
                                   (size_t)rloc * ld + lig * 4;
                    Unit<TD> so[CPL], yo[CPL];
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        if (c * L + lig < Q) {
                            so[c].load(sS + c * L * 4);
                            yo[c].load(sY + c * L * 4);
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e) { so[c].v[e] = 0; yo[c].v[e] = 0; }
                        }
                    }
                    PA* q = accq + PU_FIXED + PU_PER_OLD * t;
                    q[0] += dot_units<AD>(sn, yo);
                    q[1] += dot_units<AD>(so, yn);
                    q[2] += dot_units<AD>(yn, yo);
                }
            }
        }
        // stage s is consumed: refill it with the tile kTmaStages ahead
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_async_shared();
            issue(j + kTmaStages);
        }
    }
    block_partials<PU_N>(accq, part);
}

}  // namespace lorads
