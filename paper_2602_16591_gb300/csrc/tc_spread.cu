// Alg. 2 step 1 (spreading) on the fifth-generation tensor cores, float32 plans.
//
// Per tile of T^3 stencil-start bins the spread values form a contraction over the tile's particles,
//     S[(y, z), x] = sum_p A[(y, z), p] B[p, x],   A[(y, z), p] = rho_p w_y(p, y) w_z(p, z),
//                                                  B[p, x] = w_x(p, x),
// over the tile's extended block (E = T + P - 1 points per axis; w_d(p, .) is zero outside the P
// points of particle p's stencil).  The kernel builds A and B in shared memory for 16 particles at a
// time, and one thread issues tcgen05.mma (kind::tf32, M = 128 rows of (y, z), N = 32 columns of x,
// K = 8 particles per instruction) into tensor memory.  TF32 keeps 10 mantissa bits, so every operand
// is split into a TF32 head and the float32 remainder and the product is taken as
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo term is ~2^-22 relative): float32-level
// accuracy from three tensor-core products.  Each round of 16 particles starts a fresh accumulator in
// tensor memory, adds the small cross terms first and the large A_hi B_hi products last, and is read
// back (tcgen05.ld) and summed on the CUDA cores: the float32 accumulation in tensor memory is not
// round-to-nearest, and a whole tile summed there left a relative bias of ~5e-7 in the grid (energy
// errors of ~5e-6); short rounds bring both to the level of the CUDA-core kernel.  The tile's sums
// plus the planes carried along its x-chain are written in the slab layout of k_spread (heads per
// tile, tails per chain), so k_halo is shared by both kernels.
//
// Synchronisation: MMA completion is signalled by tcgen05.commit on an mbarrier; every wait on it is
// bounded and its outcome made block-uniform (__syncthreads_or) before it steers control flow.  A wait
// that runs out sets err_flag, and the CTA waits (bounded again) for its MMAs before it frees its
// tensor memory and returns.
#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"
#include "tc_spread.h"

namespace pswf {
namespace {

// ---- PTX wrappers (tcgen05, mbarrier) --------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (K-major, no swizzle): start address, leading-dimension byte offset
// (between core matrices adjacent along K), stride-dimension byte offset (between 8-row groups),
// descriptor version 1 in bits 46-47, base offset 0, layout type 0 (no swizzle) in bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D float32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, int ncols) {   // one full warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {   // one full warp
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {   // one full warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {   // arrives on bar when the issued MMAs complete
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase `parity` of bar for at most max_cycles SM clocks; true for every thread of the
// block if it completed in time for all of them (block-uniform: the result may steer control flow that
// contains __syncthreads).
__device__ __forceinline__ bool mbar_wait_block(uint64_t* bar, uint32_t parity, long long max_cycles) {
    const long long t0 = clock64();
    bool ok = mbar_test(bar, parity);
    while (!ok && clock64() - t0 < max_cycles) ok = mbar_test(bar, parity);
    return !__syncthreads_or(!ok);
}

// 32 consecutive float32 columns of this thread's tensor-memory lane (warp-collective).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Columns 0..19 of this thread's tensor-memory lane (x16 + x4 loads, warp-collective).
__device__ __forceinline__ void tmem_ld20(uint32_t taddr, float (&v)[20]) {
    uint32_t r[20];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19])
                 : "r"(taddr + 16));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 20; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 head of a float32 value (round to nearest, ties away: cvt.rna.tf32.f32) and its remainder.
__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    hi = __uint_as_float(h);
    lo = v - hi;
}


constexpr int kTcChunk = 16;   // particles per round of MMAs (the K extent of A and B)
constexpr int kTcN = 32;       // accumulator columns (x), E <= 32
constexpr int kTcRowBytes = kTcChunk * 4;                // one operand row: kTcChunk float32 values
constexpr int kTcSBO = (kTcChunk / 4) * 128;             // 8-row groups: kTcChunk / 4 core matrices of 128 B
constexpr int kTcLBO = 128;                              // core matrices adjacent along K
constexpr long long kTcWaitCycles = 2000000000ll;        // ~1 s at 2 GHz per mbarrier wait

// Canonical K-major, no-swizzle position (in floats) of element (row, k) of an operand with kTcChunk
// K-values per row: core matrices of 8 rows x 4 values (16 B per row, 128 B each), K-adjacent core
// matrices 128 B apart, 8-row groups kTcSBO apart.
__device__ __forceinline__ int kmajor(int row, int k) {
    return (((row >> 3) * (kTcChunk / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4) >> 2;
}

template <int P>
__global__ void __launch_bounds__(128 * tc_spread_mblocks(P), tc_spread_mblocks(P) <= 3 ? 3 : 2) k_spread_tc(
    const Vec4<float>* __restrict__ rec, const int2* __restrict__ idx, const int* __restrict__ tile_off,
    const float* __restrict__ wcoef, int degw, SpreadChain ch, float* __restrict__ scratch, int* __restrict__ err_flag) {
    constexpr int T = kTile32, E = T + P - 1, ET = E - T, NMB = tc_spread_mblocks(P), NT = 128 * NMB;
    constexpr int EP = (E + 3) / 4 * 4, COLS = tc_spread_tmem_cols(P);
    constexpr int ABYTES = 128 * NMB * kTcRowBytes;   // one of A_hi, A_lo
    static_assert(E <= kTcN && E * E <= 128 * NMB, "tile block exceeds the accumulator shape");
    constexpr int NLD = E <= 20 ? 20 : 32;   // accumulator columns read back per round
    auto tmem_ld_cols = [](uint32_t taddr, float (&v)[NLD]) {
        if constexpr (NLD == 20) tmem_ld20(taddr, v); else tmem_ld32(taddr, v);
    };
    extern __shared__ __align__(1024) unsigned char smem[];
    float* Ahi = reinterpret_cast<float*>(smem);
    float* Alo = reinterpret_cast<float*>(smem + ABYTES);
    float* Bhi = reinterpret_cast<float*>(smem + 2 * ABYTES);
    float* Blo = Bhi + kTcN * kTcChunk;
    // window weights of a round, two buffers (the next round's are computed while the MMAs run):
    // w_x(p, x) for x < kTcN, rho_p w_y(p, y) and w_z(p, z) for y, z < EP, zero outside the stencil
    constexpr int WROUND = kTcChunk * (kTcN + 2 * EP);
    float* Wbuf = Blo + kTcN * kTcChunk;
    float* sc = Wbuf + 2 * WROUND;       // window polynomials
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5;
    for (int i = t; i < P * (degw + 1); i += NT) sc[i] = wcoef[i];
    for (int i = t; i < 2 * ABYTES / 16; i += NT) reinterpret_cast<float4*>(smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (warp == 0) {
        tmem_alloc(&tmem_base, COLS);
        tmem_relinquish();
    }
    if (t == 0) mbar_init(&bar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base;

    const int qx = blockIdx.x / ch.nyz, rem = blockIdx.x - qx * ch.nyz;   // this chain: tiles (qx K + k, rem)
    const int row = t;                                                  // (y, z) row of S owned by this thread
    const bool own = row < E * E;
    const int y = row / E, z = row - (row / E) * E;
    const uint32_t lane_addr = tbase + (static_cast<uint32_t>((warp & 3) * 32) << 16) + (warp >> 2) * kTcN;
    constexpr uint32_t idesc = idesc_tf32(128, kTcN);
    // descriptors of the operand bases (every MMA adds its offset to the 14-bit address field; the
    // operands end below 256 KB of shared memory, so the field does not overflow)
    const uint64_t dAhi = smem_desc(smem_addr(Ahi), kTcLBO, kTcSBO), dAlo = smem_desc(smem_addr(Alo), kTcLBO, kTcSBO);
    const uint64_t dBhi = smem_desc(smem_addr(Bhi), kTcLBO, kTcSBO), dBlo = smem_desc(smem_addr(Blo), kTcLBO, kTcSBO);
    float carry[ET];
#pragma unroll
    for (int a = 0; a < ET; ++a) carry[a] = 0.f;
    float* heads = scratch;
    float* tails = scratch + static_cast<size_t>(ch.ntiles) * T * E * E;
    uint32_t phase = 0;
    bool failed = false;

    for (int k = 0; k < ch.K && !failed; ++k) {
        const int tile = (qx * ch.K + k) * ch.nyz + rem;
        const int beg = tile_off[tile], end = tile_off[tile + 1];
        float tacc[E];
#pragma unroll
        for (int a = 0; a < E; ++a) tacc[a] = 0.f;
        // window weights of the round starting at `first` into buffer b: task (particle j, axis d) per
        // thread writes the whole zero-padded row (16-byte stores, then the P values of the stencil)
        auto weights = [&](int first, int b) {
            if (t < 3 * kTcChunk) {
                const int j = t / 3, d = t - 3 * j, len = d == 0 ? kTcN : EP;
                float* W = Wbuf + b * WROUND + (d == 0 ? j * kTcN : kTcChunk * kTcN + ((d - 1) * kTcChunk + j) * EP);
                for (int e = 0; e < len; e += 4) *reinterpret_cast<float4*>(W + e) = make_float4(0.f, 0.f, 0.f, 0.f);
                if (first + j < end) {
                    const Vec4<float> r = rec[first + j];
                    const int o = (idx[first + j].x >> (8 * d)) & 0xff;
                    float w[P];
                    window_weights<float, P>(sc, degw, d == 0 ? r.x : (d == 1 ? r.y : r.z), w);
                    const float scale = d == 1 ? r.w : 1.f;
#pragma unroll
                    for (int a = 0; a < P; ++a) W[o + a] = w[a] * scale;
                }
            }
        };
        if (beg < end) weights(beg, 0);
        __syncthreads();
        int rb = 0;   // weight buffer of the current round
        for (int base = beg; base < end && !failed; base += kTcChunk, rb ^= 1) {
            const float* Wx = Wbuf + rb * WROUND;
            const float* Wy = Wx + kTcChunk * kTcN;
            const float* Wz = Wy + kTcChunk * EP;
            // (1) operands: A[(y, z), p] = rho_p w_y(p, y) w_z(p, z) (row of this thread) and B[x, p] = w_x(p, x)
            //     (all threads), split into TF32 head and remainder
            if (own) {
#pragma unroll
                for (int p0 = 0; p0 < kTcChunk; p0 += 4) {
                    float v[4], hi[4], lo[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        v[q] = Wy[(p0 + q) * EP + y] * Wz[(p0 + q) * EP + z];
                        split_tf32(v[q], hi[q], lo[q]);
                    }
                    *reinterpret_cast<float4*>(Ahi + kmajor(row, p0)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<float4*>(Alo + kmajor(row, p0)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
            for (int e = t; e < kTcN * kTcChunk; e += NT) {
                const int j = e / kTcN, x = e - j * kTcN;
                float hi, lo;
                split_tf32(Wx[j * kTcN + x], hi, lo);
                Bhi[kmajor(x, j)] = hi;
                Blo[kmajor(x, j)] = lo;
            }
            fence_async_smem();   // generic-proxy stores of A and B -> visible to the tensor cores
            __syncthreads();
            // (2) one thread issues the MMAs of the round: D[mb] = A_hi B_hi + A_hi B_lo + A_lo B_hi.
            // Every round starts a fresh accumulator: the two cross terms of each K step first, the
            // A_hi B_hi products last, so tensor memory accumulates few terms and the large ones last
            // (its float32 accumulation is not round-to-nearest: summing a whole tile there left a
            // relative bias of ~5e-7 in the grid); the rounds are added on the CUDA cores.
            if (t == 0) {
                tc_fence_after();
#pragma unroll
                for (int mb = 0; mb < NMB; ++mb) {
                    const uint32_t d = tbase + mb * kTcN;
#pragma unroll
                    for (int ks = 0; ks < kTcChunk / 8; ++ks) {   // 8 particles (two core matrices) per MMA
                        // operand offsets enter the descriptors' address field (bytes / 16)
                        const uint64_t ao = (mb * 16 * kTcSBO + ks * 2 * kTcLBO) >> 4, bo = (ks * 2 * kTcLBO) >> 4;
                        mma_tf32(d, dAlo + ao, dBhi + bo, idesc, ks > 0 ? 1u : 0u);
                        mma_tf32(d, dAhi + ao, dBlo + bo, idesc, 1u);
                    }
#pragma unroll
                    for (int ks = 0; ks < kTcChunk / 8; ++ks) {
                        const uint64_t ao = (mb * 16 * kTcSBO + ks * 2 * kTcLBO) >> 4, bo = (ks * 2 * kTcLBO) >> 4;
                        mma_tf32(d, dAhi + ao, dBhi + bo, idesc, 1u);
                    }
                }
                mma_commit(&bar);
            }
            // (3) while the MMAs run: the next round's window weights into the other buffer
            if (base + kTcChunk < end) weights(base + kTcChunk, rb ^ 1);
            // (4) the round's MMAs complete before A and B are rebuilt or S is read (the wait is also the
            //     barrier that publishes the next round's weights)
            if (!mbar_wait_block(&bar, phase, kTcWaitCycles)) failed = true;
            phase ^= 1u;
            if (failed) break;
            // (5) the round's sums into the tile's accumulators (round to nearest)
            tc_fence_after();
            float sv[NLD];
            tmem_ld_cols(lane_addr, sv);
#pragma unroll
            for (int a = 0; a < E; ++a) tacc[a] += sv[a];
            tc_fence_before();   // loads done before the next round's MMAs (ordered by its __syncthreads)
        }
        if (failed) break;
        // epilogue: the tile's sums (+ the planes carried along the chain); heads out, the rest carried on
        if (own) {
            float* out = heads + static_cast<size_t>(tile) * T * E * E;
#pragma unroll
            for (int a = 0; a < T; ++a) out[a * E * E + row] = tacc[a] + (a < ET ? carry[a] : 0.f);
#pragma unroll
            for (int a = 0; a < ET; ++a) carry[a] = tacc[a + T] + (a + T < ET ? carry[a + T] : 0.f);
        }
    }
    if (!failed && own) {   // the chain's tail: planes that belong to the tiles after the chain
        float* out = tails + static_cast<size_t>(blockIdx.x) * ET * E * E;
#pragma unroll
        for (int a = 0; a < ET; ++a) out[a * E * E + row] = carry[a];
    }
    if (failed) {   // let the outstanding MMAs finish (bounded) before the tensor memory is released
        if (t == 0) atomicExch(err_flag, 1);
        mbar_wait_block(&bar, phase ^ 1u, kTcWaitCycles);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, COLS);
}

template <int P>
cudaError_t spread_tc_p(int ntiles, const Vec4<float>* rec, const int2* idx, const int* tile_off, const float* wcoef,
                        int degw, SpreadChain ch, float* scratch, int* err_flag, cudaStream_t s) {
    const size_t smem = tc_spread_smem(P, degw);
    auto kern = k_spread_tc<P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<ntiles / ch.K, 128 * tc_spread_mblocks(P), smem, s>>>(rec, idx, tile_off, wcoef, degw, ch, scratch, err_flag);
    return cudaGetLastError();
}

// The bounded wait on a barrier that nothing arrives at (the timeout path, exercised by a test):
// flag = 1 when the wait ran out after max_cycles SM clocks.
__global__ void k_wait_probe(long long max_cycles, int* __restrict__ flag) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool ok = mbar_wait_block(&bar, 0u, max_cycles);
    if (threadIdx.x == 0) *flag = ok ? 0 : 1;
}

}  // namespace

bool tc_spread_supports(int P) { return P >= 3 && P <= 14; }

size_t tc_spread_smem(int P, int degw) {
    const int E = kTile32 + P - 1, EP = (E + 3) / 4 * 4;
    return 2 * static_cast<size_t>(128) * tc_spread_mblocks(P) * kTcRowBytes + 2 * sizeof(float) * kTcN * kTcChunk +
           2 * sizeof(float) * kTcChunk * (kTcN + 2 * EP) + sizeof(float) * P * (degw + 1);
}

cudaError_t launch_spread_tc(int P, int ntiles, const Vec4<float>* rec, const int2* idx, const int* tile_off,
                             const float* wcoef, int degw, SpreadChain ch, float* scratch, int* err_flag, cudaStream_t s) {
    switch (P) {
#define PSWF_TC_CASE(PP) \
    case PP: return spread_tc_p<PP>(ntiles, rec, idx, tile_off, wcoef, degw, ch, scratch, err_flag, s);
        PSWF_TC_CASE(3) PSWF_TC_CASE(4) PSWF_TC_CASE(5) PSWF_TC_CASE(6) PSWF_TC_CASE(7) PSWF_TC_CASE(8)
        PSWF_TC_CASE(9) PSWF_TC_CASE(10) PSWF_TC_CASE(11) PSWF_TC_CASE(12) PSWF_TC_CASE(13) PSWF_TC_CASE(14)
#undef PSWF_TC_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wait_probe(long long max_cycles, int* flag, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(max_cycles, flag);
    return cudaGetLastError();
}

}  // namespace pswf
