// btrt_tma.cuh -- TMA-staged sweep for FP32 compute with FP32/FP16/BF16 storage.
//
// A persistent block walks tiles of TX x TY nodes.  For each tile one 3-D TMA
// copy brings the nine input planes (TX + 2 PAD) x (TY + 2) around the tile into
// shared memory (the halo covers every streaming shift; PAD keeps the copy's x
// origin on a 16-byte boundary), tracked by an mbarrier; two stages alternate so
// the next tile's copy overlaps this tile's collisions.  Each thread pulls its
// nodes' populations from shared memory at compile-time offsets, collides, and
// writes the post-collision populations into an output tile that one 3-D TMA
// store sends back to global memory (clipped at the grid edge).  Nodes on the
// domain boundary take the ordinary global-memory path with periodic wrap or
// bounce-back.  With the local storage shift the neighbours' phi^{n-1} values
// come through L1 from the previous phi plane.  Every mbarrier wait is bounded; on expiry the block raises flag
// bit 2, waits (bounded) for its own copies and returns.
#pragma once

#include <cuda.h>

#include "btrt_sweep.cuh"

namespace btrt {

template <typename S> struct TmaTile;
template <> struct TmaTile<__half> { static constexpr int TX = 64, TY = 16, PAD = 8; };
template <> struct TmaTile<__nv_bfloat16> { static constexpr int TX = 64, TY = 16, PAD = 8; };
template <> struct TmaTile<float> { static constexpr int TX = 32, TY = 16, PAD = 4; };

template <typename S> struct TmaGeom {
    static constexpr int TX = TmaTile<S>::TX, TY = TmaTile<S>::TY, PAD = TmaTile<S>::PAD;
    static constexpr int BX = TX + 2 * PAD, BY = TY + 2;
    static constexpr int IN_BYTES = 9 * BY * BX * (int)sizeof(S);
    static constexpr int IN_STAGE = (IN_BYTES + 127) / 128 * 128;
    static constexpr int OUT_BYTES = 9 * TY * TX * (int)sizeof(S);
    static constexpr int OUT_STAGE = (OUT_BYTES + 127) / 128 * 128;
    // + mbarriers and a flag (128 B) + room to align the base to 128 B
    static constexpr int SMEM = 2 * IN_STAGE + OUT_STAGE + 128 + 128;
    static constexpr int THREADS = 256;
    static constexpr int ROWS = TY / (THREADS / TX);              // nodes per thread
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on an mbarrier phase; false when the bound was reached
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t k = 0; k < limit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

template <typename S, int SH, int MODE, int SRC>
__global__ void __launch_bounds__(256) sweep_tma_kernel(const __grid_constant__ SweepParams<float> p,
                                                        const __grid_constant__ CUtensorMap in_map,
                                                        const __grid_constant__ CUtensorMap out_map, int ntx,
                                                        int ntiles, uint32_t wait_limit) {
    using G = TmaGeom<S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations and sources start on 128-byte boundaries
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    auto in_tile = [&](int s) { return reinterpret_cast<S *>(smem + s * G::IN_STAGE); };
    S *out_tile = reinterpret_cast<S *>(smem + 2 * G::IN_STAGE);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * G::IN_STAGE + G::OUT_STAGE);
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    const int tid = threadIdx.x;
    const int lx = tid % G::TX;
    const int ly0 = tid / G::TX;
    constexpr int YSTEP = G::THREADS / G::TX;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            const int t = blockIdx.x + s * gridDim.x;
            if (t < ntiles) {
                mbar_expect_tx(&bar[s], G::IN_BYTES);
                tma_load_3d(in_tile(s), &in_map, (t % ntx) * G::TX - G::PAD, (t / ntx) * G::TY - 1, 0, &bar[s]);
            }
        }
    }
    uint32_t phase0 = 0u, phase1 = 0u;   // parity to wait for on each stage's mbarrier
    int &failed = *reinterpret_cast<int *>(bar + 2);
    for (int j = 0;; ++j) {
        const int t = blockIdx.x + j * gridDim.x;
        if (t >= ntiles) break;
        const int s = j & 1;
        const bool ok = mbar_wait(&bar[s], s ? phase1 : phase0, wait_limit);
        if (tid == 0) {
            failed = ok ? 0 : 1;
            bulk_wait_read_all();   // the previous output tile has been read out
        }
        __syncthreads();
        if (__syncthreads_or(!ok) || failed) {
            if (tid == 0) {
                atomicOr(p.flags, 4);
                // give the outstanding copies of both stages a bounded chance to land, then leave
                mbar_wait(&bar[0], phase0, wait_limit);
                mbar_wait(&bar[1], phase1, wait_limit);
                bulk_wait_all();
            }
            return;
        }
        if (s) phase1 ^= 1u; else phase0 ^= 1u;
        const int x0 = (t % ntx) * G::TX, y0 = (t / ntx) * G::TY;
        const S *tin = in_tile(s);
        const int x = x0 + lx;
        float xs = 0.f, xc = 0.f;
        if (SRC == 2 && x < p.nx) {
            xs = p.Xs[BTRT_IX(p.flags, x, p.nx)];
            xc = p.Xc[BTRT_IX(p.flags, x, p.nx)];
        }
#pragma unroll 1
        for (int r = 0; r < G::ROWS; ++r) {
            const int ly = ly0 + r * YSTEP;
            const int y = y0 + ly;
            if (x >= p.nx || y >= p.ny) continue;
            const int node = y * p.pitch + x;
            float f[9];
            const float phi_prev = p.phi_in[BTRT_IX(p.flags, node, p.plane)];
            if (x > 0 && x < p.nx - 1 && y > 0 && y < p.ny - 1) {
                const S *base = tin + (ly + 1) * G::BX + (lx + G::PAD);
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = Storage<S>::load(base[i * G::BY * G::BX - ey_of(i) * G::BX - ex_of(i)]);
                if constexpr (SH == kShiftLocal) {
#pragma unroll
                    for (int i = 1; i < 9; ++i)
                        f[i] = fma(wgt<float>(i),
                                   p.phi_in[BTRT_IX(p.flags, node - ey_of(i) * p.pitch - ex_of(i), p.plane)] - phi_prev,
                                   f[i]);
                }
            } else {
                pull_boundary<float, S, SH, false>(p, fin, x, y, node, phi_prev, f);
            }
            const float src = source_at<float, SRC>(p, xs, xc, y, node);
            const float rs = SH == kShiftLocal ? phi_prev : p.phi_ref;
            float phid;
            const float phi = collide_fold<float, MODE, SRC, SH>(p, f, rs, phi_prev, src, false, node, phid);
            S *o = out_tile + ly * G::TX + lx;
#pragma unroll
            for (int i = 0; i < 9; ++i) o[i * G::TY * G::TX] = store_value<float, S, SH>(i, f[i], phid);
            p.phi_out[BTRT_IX(p.flags, node, p.plane)] = phi;
            if (not_finite(phi)) atomicOr(p.flags, 1);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&out_map, out_tile, x0, y0, 0);
            bulk_commit();
            const int tn = blockIdx.x + (j + 2) * gridDim.x;
            if (tn < ntiles) {
                mbar_expect_tx(&bar[s], G::IN_BYTES);
                tma_load_3d(in_tile(s), &in_map, (tn % ntx) * G::TX - G::PAD, (tn / ntx) * G::TY - 1, 0, &bar[s]);
            }
        }
    }
    if (tid == 0) bulk_wait_all();
}

}  // namespace btrt
