// Device kernels of the PSWF fast Ewald pipeline (sm_103a).
//
// Pipeline per evaluation (paper: Alg. 2 plus the real-space sum of Sec. 3.1.1):
//   k_prep     wrap x into [0,L)^3, spreading-tile and real-space-cell keys, ranks (counting sort 1/3)
//   k_scan     exclusive scan of the per-tile and per-cell counts          (counting sort 2/3)
//   k_scatter  sorted particle records (per-tile window offsets, per-cell local coords) (3/3)
//   k_spread   Alg. 2 step 1: per-tile spreading into register-held grid columns (no atomics)
//   k_halo     sums the overlapping tile blocks into the periodic grid (halo accumulation)
//   cuFFT R2C  Alg. 2 step 2
//   k_scale    Alg. 2 step 3: b_k = S(k) a_k with S from host tables
//   cuFFT C2R  Alg. 2 step 4
//   k_interp   Alg. 2 step 5 and eq. force: phi^far, grad phi^far; writes phi - self, F
//   k_short    real-space sum of the residual R (eq. R) over the cell list (second stream, concurrent
//              with spread..interp), into separate phi/F buffers
//   k_combine_energy  phi += phi_sr, F += F_sr, E = 1/2 sum rho phi (Remark on energy); its last block
//              adds the block sums
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <type_traits>

#include "ff.cuh"

namespace pswf {

template <typename real> struct alignas(4 * sizeof(real)) Vec4 { real x, y, z, w; };

// Geometry and sizes shared by the kernels of one plan (passed by value).  Per-axis arrays (x, y, z)
// describe cuboid boxes (Remark on cuboid domains, Sec. 6.1); a cube has three equal entries.
struct Geom {
    int n, P, T, reach, degw, degr;
    int reachz;   // real-space cells per cutoff radius along z (reach along x and y)
    int K;        // spreading tiles per x-chain (a divisor of nt[0]; k_spread)
    int m[3], nt[3], ncell[3];
    double L[3], invL[3], invh[3], cellw[3], invcellw[3];
    double rc, self;
    // float-float (hi, lo) copies of L, 1/L, 1/h, cell width and its inverse for locate_ff
    float Lf[3][2], invLf[3][2], invhf[3][2], cellwf[3][2], invcellwf[3][2];
};

// Spreading / interpolation tile edge (grid points); m is a multiple of it.  float32 plans use 8 (the
// extended blocks of neighbouring tiles overlap (1 + (P-1)/8)^3 times instead of (1 + (P-1)/4)^3, and
// an interpolation block serves ~8x more particles per staged grid block); float64 and float-float
// plans, whose extended blocks are twice as large per value, use 4.
constexpr int kTile32 = 8, kTile64 = 4;
template <typename real>
constexpr int spread_tile() { return sizeof(real) == 4 ? kTile32 : kTile64; }

// Everything a particle needs, computed once from its position (float64).
struct Located {
    double w[3];     // wrapped position in [0, L)
    double z[3];     // window coordinate z = 2 (x/h - l0) - (P - 1) in (-1, 1]
    int lw[3];       // stencil start l0 mod m
    int cell[3];     // real-space cell
    double loc[3];   // position relative to the cell origin
    bool finite;
};

__device__ inline Located locate(const double* xp, const Geom& g) {
    Located r;
    r.finite = true;
    for (int d = 0; d < 3; ++d) {
        double x = xp[d];
        if (!isfinite(x)) { r.finite = false; x = 0.0; }
        double w = x - g.L[d] * floor(x * g.invL[d]);
        if (w >= g.L[d]) w -= g.L[d];
        if (w < 0.0) w = 0.0;
        r.w[d] = w;
        const double t = w * g.invh[d];
        const int l0 = static_cast<int>(ceil(t - 0.5 * g.P));
        r.z[d] = 2.0 * (t - l0) - (g.P - 1);
        int lw = l0 % g.m[d];
        if (lw < 0) lw += g.m[d];
        r.lw[d] = lw;
        int c = static_cast<int>(w * g.invcellw[d]);   // no float64 division: multiply, then clamp
        c = c < 0 ? 0 : (c >= g.ncell[d] ? g.ncell[d] - 1 : c);
        r.cell[d] = c;
        r.loc[d] = w - c * g.cellw[d];
    }
    return r;
}

// locate() in float-float arithmetic for the float32 plans, whose records are float32 (z) and
// float-float (local coordinates): each coordinate is split once into hi + lo floats (~48 bits), then
// wrapping, stencil start, window coordinate and cell use float32 operations only.  GB300 issues
// float64 at ~1/64 of the float32 rate, and the float64 locate() made the sort kernels FP64-bound.
// Positions more than 2^22 box lengths from the origin take the float64 route.
struct LocatedF {
    float z[3];      // window coordinate
    int lw[3];       // stencil start l0 mod m
    int cell[3];     // real-space cell
    ff loc[3];       // position relative to the cell origin (normalised hi + lo)
    bool finite;
};

__device__ __forceinline__ ff ff_c(const float (&v)[2]) { return ff{v[0], v[1]}; }

// floor / ceil of a normalised float-float value (|l| <= ulp(h)/2: only an integral h can be moved)
__device__ __forceinline__ float ff_floor(ff a) {
    const float f = floorf(a.h);
    return f == a.h ? f - (a.l < 0.f ? 1.f : 0.f) : f;
}
__device__ __forceinline__ float ff_ceil(ff a) {
    const float c = ceilf(a.h);
    return c == a.h ? c + (a.l > 0.f ? 1.f : 0.f) : c;
}

__device__ inline LocatedF locate_ff(const double* xp, const Geom& g) {
    LocatedF r;
    r.finite = true;
    for (int d = 0; d < 3; ++d) {
        double x = xp[d];
        if ((__double2hiint(x) & 0x7ff00000) == 0x7ff00000) { r.finite = false; x = 0.0; }
        const ff L = ff_c(g.Lf[d]);
        ff w = ff_from_double(x);
        const bool inside = (w.h > 0.f || (w.h == 0.f && w.l >= 0.f)) && (w.h < L.h || (w.h == L.h && w.l < L.l));
        if (!inside) {
            const ff u = ff_mul(w, ff_c(g.invLf[d]));
            if (fabsf(u.h) < 4194304.f) {
                w = ff_sub(w, ff_mul_f(L, ff_floor(u)));
            } else {   // far outside the box: float64 reduction
                const double wd = x - g.L[d] * floor(x * g.invL[d]);
                w = ff_from_double(wd);
            }
            if (w.h < 0.f || (w.h == 0.f && w.l < 0.f)) w = ff_add(w, L);
            if (w.h > L.h || (w.h == L.h && w.l >= L.l)) w = ff_sub(w, L);
            if (w.h < 0.f || (w.h == 0.f && w.l < 0.f)) w = ff{0.f, 0.f};
        }
        const ff t = ff_mul(w, ff_c(g.invhf[d]));
        const float l0 = ff_ceil(ff_add(t, ff_make(-0.5f * g.P)));
        const ff dt = ff_sub(t, ff_make(l0));                    // in (P/2 - 1, P/2]
        r.z[d] = __fadd_rn(__fmaf_rn(2.f, dt.h, static_cast<float>(1 - g.P)), __fmul_rn(2.f, dt.l));
        int lw = static_cast<int>(l0) % g.m[d];
        if (lw < 0) lw += g.m[d];
        r.lw[d] = lw;
        int c = static_cast<int>(ff_floor(ff_mul(w, ff_c(g.invcellwf[d]))));
        c = c < 0 ? 0 : (c >= g.ncell[d] ? g.ncell[d] - 1 : c);
        r.cell[d] = c;
        r.loc[d] = ff_sub(w, ff_mul_f(ff_c(g.cellwf[d]), static_cast<float>(c)));
    }
    return r;
}

template <typename Loc>
__device__ inline int tile_of(const Loc& r, const Geom& g) {
    return ((r.lw[0] / g.T) * g.nt[1] + r.lw[1] / g.T) * g.nt[2] + r.lw[2] / g.T;
}
template <typename Loc>
__device__ inline int cell_of(const Loc& r, const Geom& g) {
    return (r.cell[0] * g.ncell[1] + r.cell[1]) * g.ncell[2] + r.cell[2];
}

// status[0] = sum rho, status[1] = sum |rho|, status[2] = number of non-finite inputs.
// FFLOC: locate in float-float (float32 plans) instead of float64; k_scatter of the same plan must use
// the same routine (the keys and ranks written here place its records).
template <bool FFLOC>
__device__ __forceinline__ void k_prep_body(int bx, const double* __restrict__ x, const double* __restrict__ rho, Geom g,
                                              int* __restrict__ key_rank, int* __restrict__ tile_cnt,
                                              int* __restrict__ cell_cnt, double* __restrict__ status) {
    const int i = bx * blockDim.x + threadIdx.x;
    double q = 0.0;
    int bad = 0;
    if (i < g.n) {
        q = rho[i];
        if ((__double2hiint(q) & 0x7ff00000) == 0x7ff00000) { bad = 1; q = 0.0; }
        int t, c;
        if constexpr (FFLOC) {
            const LocatedF r = locate_ff(x + 3 * static_cast<size_t>(i), g);
            if (!r.finite) bad = 1;
            t = tile_of(r, g);
            c = cell_of(r, g);
        } else {
            const Located r = locate(x + 3 * static_cast<size_t>(i), g);
            if (!r.finite) bad = 1;
            t = tile_of(r, g);
            c = cell_of(r, g);
        }
        const int rt = atomicAdd(tile_cnt + t, 1);
        const int rc = atomicAdd(cell_cnt + c, 1);
        reinterpret_cast<int4*>(key_rank)[i] = make_int4(t, rt, c, rc);
    }
    // block sums of the neutrality diagnostics: staged in shared memory and added by one warp, so the
    // float64 additions run once per 8 values instead of in every lane's shuffle tree
    __shared__ double red[256];
    __shared__ int nbad;
    if (threadIdx.x == 0) nbad = 0;
    red[threadIdx.x] = q;
    __syncthreads();
    if (bad) atomicAdd(&nbad, 1);
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        double sq = 0.0, sa = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const double v = red[lane + 32 * k];
            sq += v;
            sa += fabs(v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
        }
        __syncwarp();
        if (lane == 0) {
            atomicAdd(status + 0, sq);
            atomicAdd(status + 1, sa);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && nbad > 0) atomicAdd(status + 2, static_cast<double>(nbad));
}

template <bool FFLOC>
__global__ void __launch_bounds__(256) k_prep(const double* __restrict__ x, const double* __restrict__ rho, Geom g,
                                              int* __restrict__ key_rank, int* __restrict__ tile_cnt,
                                              int* __restrict__ cell_cnt, double* __restrict__ status) {
    k_prep_body<FFLOC>(blockIdx.x, x, rho, g, key_rank, tile_cnt, cell_cnt, status);
}

// Exclusive scan of cnt[0..N) into off[0..N]; one block per segment (blockIdx.x = 0 / 1).
__device__ __forceinline__ void k_scan_body(int bx, const int* __restrict__ cnt0, int* __restrict__ off0, int n0,
                                               const int* __restrict__ cnt1, int* __restrict__ off1, int n1) {
    const int* cnt = bx == 0 ? cnt0 : cnt1;
    int* off = bx == 0 ? off0 : off1;
    const int N = bx == 0 ? n0 : n1;
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int carry = 0;
    constexpr int ITEMS = 16;   // 16K counters per round: the ~3e4 cell counters of a 1e5-particle plan in 2 rounds
    for (int base = 0; base < N; base += blockDim.x * ITEMS) {
        int v[ITEMS], s = 0;
        const int i0 = base + threadIdx.x * ITEMS;
        if (i0 + ITEMS <= N) {   // whole 64-byte runs: vector loads (the arrays are cudaMalloc-aligned)
            const int4* c4 = reinterpret_cast<const int4*>(cnt + i0);
#pragma unroll
            for (int q = 0; q < ITEMS / 4; ++q) {
                const int4 t = c4[q];
                v[4 * q] = t.x;
                v[4 * q + 1] = t.y;
                v[4 * q + 2] = t.z;
                v[4 * q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < ITEMS; ++k) v[k] = (i0 + k < N) ? cnt[i0 + k] : 0;
        }
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) s += v[k];
        int x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        int e = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - s;
        if (i0 + ITEMS <= N) {
            int4* o4 = reinterpret_cast<int4*>(off + i0);
#pragma unroll
            for (int q = 0; q < ITEMS / 4; ++q) {
                int4 t;
                t.x = e;
                e += v[4 * q];
                t.y = e;
                e += v[4 * q + 1];
                t.z = e;
                e += v[4 * q + 2];
                t.w = e;
                e += v[4 * q + 3];
                o4[q] = t;
            }
        } else {
#pragma unroll
            for (int k = 0; k < ITEMS; ++k) {
                if (i0 + k < N) off[i0 + k] = e;
                e += v[k];
            }
        }
        const int total = wsum[nw - 1];
        __syncthreads();
        carry += total;
    }
    if (threadIdx.x == 0) off[N] = carry;
}

static __global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ cnt0, int* __restrict__ off0, int n0,
                                               const int* __restrict__ cnt1, int* __restrict__ off1, int n1) {
    k_scan_body(blockIdx.x, cnt0, off0, n0, cnt1, off1, n1);
}

// Multi-block form of k_scan for long counter arrays (the ~1e6 tiles and cells of the 1e7-particle
// plans), in three launches without inter-block waits: k_scan_sums (one block per kScanChunk counters
// of either segment: its sum), k_scan over the block sums (their exclusive offsets, two blocks), and
// k_scan_apply (every block scans its chunk again from its offset).  Blocks [0, nb0) cover segment 0.
constexpr int kScanItems = 16, kScanChunk = 1024 * kScanItems;

// exclusive scan of the chunk cnt[i0 .. i0 + kScanChunk) of a length-N array from carry (written to off
// when off != nullptr); returns the chunk's total.  1024 threads.
__device__ __forceinline__ int scan_chunk(const int* __restrict__ cnt, int* __restrict__ off, int N, int base,
                                          int carry) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int v[kScanItems], s = 0;
    const int i0 = base + threadIdx.x * kScanItems;
    if (i0 + kScanItems <= N) {   // 64-byte runs (chunk starts are multiples of 16K counters)
        const int4* c4 = reinterpret_cast<const int4*>(cnt + i0);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const int4 t = c4[q];
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = (i0 + k < N) ? cnt[i0 + k] : 0;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const int total = wsum[31];
    if (off) {
        int e = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - s;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (i0 + k < N) off[i0 + k] = e;
            e += v[k];
        }
    }
    __syncthreads();   // wsum is reused by the caller's next chunk
    return total;
}

static __global__ void __launch_bounds__(1024) k_scan_sums(const int* __restrict__ cnt0, int n0, int nb0,
                                                           const int* __restrict__ cnt1, int n1,
                                                           int* __restrict__ bsum0, int* __restrict__ bsum1) {
    const int b = blockIdx.x, seg = b >= nb0, lb = seg ? b - nb0 : b;
    const int t = scan_chunk(seg ? cnt1 : cnt0, nullptr, seg ? n1 : n0, lb * kScanChunk, 0);
    if (threadIdx.x == 0) (seg ? bsum1 : bsum0)[lb] = t;
}

// boff0[0 .. nb0] and boff1[0 .. nb1]: exclusive block offsets of the two segments (k_scan of the sums)
static __global__ void __launch_bounds__(1024) k_scan_apply(const int* __restrict__ cnt0, int* __restrict__ off0, int n0,
                                                            int nb0, const int* __restrict__ cnt1, int* __restrict__ off1,
                                                            int n1, const int* __restrict__ boff0,
                                                            const int* __restrict__ boff1) {
    const int b = blockIdx.x, seg = b >= nb0, lb = seg ? b - nb0 : b;
    const int* boff = seg ? boff1 : boff0;
    const int N = seg ? n1 : n0;
    int* off = seg ? off1 : off0;
    scan_chunk(seg ? cnt1 : cnt0, off, N, lb * kScanChunk, boff[lb]);
    if (lb == 0 && threadIdx.x == 0) off[N] = boff[(N + kScanChunk - 1) / kScanChunk];
}

// ---- stable order inside tiles and cells (counting sort, deterministic ranks) --------------------
// k_prep's atomic ranks depend on the schedule, and so would every sum over the particles of a tile
// or cell (spreading, the real-space sum).  k_place lists each bin's particles at their atomic
// positions (perm: tile order in [0, n), cell order in [n, 2n)); k_rerank then replaces every atomic
// rank by the number of particles of the same bin with a smaller input index, so the scatter writes
// each bin in input order and an evaluation is bitwise repeatable.  The rank loop of k_rerank reads
// the bin's list once per position; consecutive positions mostly share a bin, so the loads are warp
// broadcasts (a bin of b particles costs b^2 / 32 warp loads).
__device__ __forceinline__ void k_place_body(int bx, const int* __restrict__ key_rank, int n,
                                                      const int* __restrict__ tile_off,
                                                      const int* __restrict__ cell_off, int* __restrict__ perm) {
    const int i = bx * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 kr = reinterpret_cast<const int4*>(key_rank)[i];
    perm[tile_off[kr.x] + kr.y] = i;
    perm[static_cast<size_t>(n) + cell_off[kr.z] + kr.w] = i;
}

static __global__ void __launch_bounds__(256) k_place(const int* __restrict__ key_rank, int n,
                                                      const int* __restrict__ tile_off,
                                                      const int* __restrict__ cell_off, int* __restrict__ perm) {
    k_place_body(blockIdx.x, key_rank, n, tile_off, cell_off, perm);
}

// blockIdx.y = 0: tile ranks (key_rank .x/.y), 1: cell ranks (.z/.w).  Each thread owns one position
// of the bin lists; it writes only the rank word of its own particle.
__device__ __forceinline__ void k_rerank_body(int bx, int by, int* __restrict__ key_rank, int n,
                                                       const int* __restrict__ tile_off,
                                                       const int* __restrict__ cell_off,
                                                       const int* __restrict__ perm) {
    const int p = bx * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int kind = by;
    const int* list = perm + (kind ? static_cast<size_t>(n) : 0);
    const int* off = kind ? cell_off : tile_off;
    const int i = list[p];
    const int key = key_rank[4 * static_cast<size_t>(i) + 2 * kind];
    const int s = off[key], e = off[key + 1];
    int r = 0;
    for (int q = s; q < e; ++q) r += list[q] < i ? 1 : 0;
    key_rank[4 * static_cast<size_t>(i) + 2 * kind + 1] = r;
}

static __global__ void __launch_bounds__(256) k_rerank(int* __restrict__ key_rank, int n,
                                                       const int* __restrict__ tile_off,
                                                       const int* __restrict__ cell_off,
                                                       const int* __restrict__ perm) {
    k_rerank_body(blockIdx.x, blockIdx.y, key_rank, n, tile_off, cell_off, perm);
}

// Sorted records.  Spreading side (tile order): {z0, z1, z2, rho}, {packed offsets in tile, original index}.
// Real-space side (cell order): {local x, y, z, rho}, {cell id, original index}.
template <typename real>
__device__ __forceinline__ void k_scatter_body(int bx, const double* __restrict__ x, const double* __restrict__ rho, Geom g,
                                                 const int* __restrict__ key_rank, const int* __restrict__ tile_off,
                                                 const int* __restrict__ cell_off, Vec4<real>* __restrict__ sp_rec,
                                                 int2* __restrict__ sp_idx, Vec4<real>* __restrict__ sr_rec,
                                                 int2* __restrict__ sr_idx, Vec4<real>* __restrict__ sr_lo,
                                                 float4* __restrict__ sr_f32) {
    const int i = bx * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    double q = rho[i];
    if ((__double2hiint(q) & 0x7ff00000) == 0x7ff00000) q = 0.0;
    const int4 kr = reinterpret_cast<const int4*>(key_rank)[i];
    const int ps = tile_off[kr.x] + kr.y;
    const int pc = cell_off[kr.z] + kr.w;
    if constexpr (std::is_same<real, float>::value) {
        // float32 records: the float-float locate of k_prep<true>
        const LocatedF r = locate_ff(x + 3 * static_cast<size_t>(i), g);
        const float qf = static_cast<float>(q);
        sp_rec[ps] = Vec4<float>{r.z[0], r.z[1], r.z[2], qf};
        sp_idx[ps] = make_int2((r.lw[0] % g.T) | ((r.lw[1] % g.T) << 8) | ((r.lw[2] % g.T) << 16), i);
        sr_rec[pc] = Vec4<float>{r.loc[0].h, r.loc[1].h, r.loc[2].h, qf};
        sr_idx[pc] = make_int2(r.cell[0] | (r.cell[1] << 10) | (r.cell[2] << 20), i);   // packed cell (< 1024 per axis)
        // rounding residue of the local coordinates (float-float) and the z cell index (its int bits: the
        // real-space kernel reads it back without a conversion instruction)
        sr_lo[pc] = Vec4<float>{r.loc[0].l, r.loc[1].l, r.loc[2].l, __int_as_float(r.cell[2])};
    } else {
        const Located r = locate(x + 3 * static_cast<size_t>(i), g);
        Vec4<real> a;
        a.x = static_cast<real>(r.z[0]);
        a.y = static_cast<real>(r.z[1]);
        a.z = static_cast<real>(r.z[2]);
        a.w = static_cast<real>(q);
        sp_rec[ps] = a;
        const int pack = (r.lw[0] % g.T) | ((r.lw[1] % g.T) << 8) | ((r.lw[2] % g.T) << 16);
        sp_idx[ps] = make_int2(pack, i);
        Vec4<real> b;
        b.x = static_cast<real>(r.loc[0]);
        b.y = static_cast<real>(r.loc[1]);
        b.z = static_cast<real>(r.loc[2]);
        b.w = static_cast<real>(q);
        sr_rec[pc] = b;
        sr_idx[pc] = make_int2(cell_of(r, g), i);
        if (sr_f32)    // float64 records get a float32 copy for the cutoff pre-test of the real-space sum
            sr_f32[pc] = make_float4(static_cast<float>(r.loc[0]), static_cast<float>(r.loc[1]),
                                     static_cast<float>(r.loc[2]), __int_as_float(r.cell[2]));
    }
}

template <typename real>
__global__ void __launch_bounds__(256) k_scatter(const double* __restrict__ x, const double* __restrict__ rho, Geom g,
                                                 const int* __restrict__ key_rank, const int* __restrict__ tile_off,
                                                 const int* __restrict__ cell_off, Vec4<real>* __restrict__ sp_rec,
                                                 int2* __restrict__ sp_idx, Vec4<real>* __restrict__ sr_rec,
                                                 int2* __restrict__ sr_idx, Vec4<real>* __restrict__ sr_lo,
                                                 float4* __restrict__ sr_f32) {
    k_scatter_body<real>(blockIdx.x, x, rho, g, key_rank, tile_off, cell_off, sp_rec, sp_idx, sr_rec, sr_idx, sr_lo, sr_f32);
}

// P window weights at one coordinate z by Horner (coefficients c[a*(deg+1) + k], monomials in z).
template <typename real, int P>
__device__ __forceinline__ void window_weights(const real* __restrict__ c, int deg, real z, real (&w)[P]) {
#pragma unroll
    for (int a = 0; a < P; ++a) w[a] = c[a * (deg + 1) + deg];
    for (int k = deg - 1; k >= 0; --k) {
#pragma unroll
        for (int a = 0; a < P; ++a) w[a] = fma(w[a], z, c[a * (deg + 1) + k]);
    }
}

// The same Horner sums with the coefficients stored by power: c[k * PP + a] (rows of PP >= P values,
// 16-byte aligned), so each power costs PP / VW vector loads instead of P scalar ones.  Same
// operations in the same order as window_weights, hence the same weights bit for bit.
template <typename real, int P, int PP>
__device__ __forceinline__ void window_weights_rows(const real* __restrict__ c, int deg, real z, real (&w)[P]) {
    constexpr int VW = 16 / static_cast<int>(sizeof(real));
    static_assert(PP % VW == 0 && PP >= P, "coefficient rows are whole 16-byte vectors");
    using V = typename std::conditional<sizeof(real) == 4, float4, double2>::type;
    const V* row = reinterpret_cast<const V*>(c + deg * PP);
#pragma unroll
    for (int i = 0; i < PP / VW; ++i) {
        const V t = row[i];
        if constexpr (sizeof(real) == 4) {
            if (4 * i < P) w[4 * i] = t.x;
            if (4 * i + 1 < P) w[4 * i + 1] = t.y;
            if (4 * i + 2 < P) w[4 * i + 2] = t.z;
            if (4 * i + 3 < P) w[4 * i + 3] = t.w;
        } else {
            if (2 * i < P) w[2 * i] = t.x;
            if (2 * i + 1 < P) w[2 * i + 1] = t.y;
        }
    }
    for (int k = deg - 1; k >= 0; --k) {
        row -= PP / VW;
#pragma unroll
        for (int i = 0; i < PP / VW; ++i) {
            const V t = row[i];
            if constexpr (sizeof(real) == 4) {
                if (4 * i < P) w[4 * i] = fma(w[4 * i], z, t.x);
                if (4 * i + 1 < P) w[4 * i + 1] = fma(w[4 * i + 1], z, t.y);
                if (4 * i + 2 < P) w[4 * i + 2] = fma(w[4 * i + 2], z, t.z);
                if (4 * i + 3 < P) w[4 * i + 3] = fma(w[4 * i + 3], z, t.w);
            } else {
                if (2 * i < P) w[2 * i] = fma(w[2 * i], z, t.x);
                if (2 * i + 1 < P) w[2 * i + 1] = fma(w[2 * i + 1], z, t.y);
            }
        }
    }
}

// ---- Alg. 2 step 1: spreading ------------------------------------------------------------------
// One CTA per tile of T^3 stencil-start bins.  Thread t owns the column (b, c) = (t / E, t % E) of
// the tile's extended block (E = T + P - 1 points per axis) and keeps its E values along the first
// axis in registers; every particle of the tile adds rho wy[b-oy] wz[c-oz] wx[.] to them.  The
// block is written to a per-tile scratch slab; k_halo sums overlapping slabs (no atomics anywhere).
constexpr int kSpreadChunk = 64;

// x-chains of the spreading: one CTA walks K consecutive tiles along x (nyz = nt_y nt_z tiles per
// x plane of tiles) and keeps its register columns across them, so only T planes per tile (the
// tile's head) plus E - T planes per chain (its tail) reach the slab buffer, instead of E planes per
// tile.  Slab layout: heads [tile][a < T][y < E][z < E], then tails [chain][a < E - T][y][z].
struct SpreadChain {
    int K, nyz, ntiles;
};

template <int P, int T>
constexpr int spread_threads() { return (((T + P - 1) * (T + P - 1) + 31) / 32) * 32; }

template <typename real, int P>
__device__ __forceinline__ void k_spread_body(int bx, const Vec4<real>* __restrict__ rec, const int2* __restrict__ idx,
                                                 const int* __restrict__ tile_off, const real* __restrict__ wcoef,
                                                 int degw, SpreadChain ch, real* __restrict__ scratch) {
    constexpr int T = spread_tile<real>(), E = T + P - 1, CH = kSpreadChunk;
    const int qx = bx / ch.nyz, rem = bx - qx * ch.nyz;   // this chain: tiles (qx K + k, rem)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // weight rows padded to whole 16-byte vectors so a thread reads a particle's P x-weights with
    // PP / VW broadcast vector loads instead of P scalar ones
    constexpr int VW = 16 / static_cast<int>(sizeof(real)), PP = (P + VW - 1) / VW * VW;
    using V = typename std::conditional<sizeof(real) == 4, float4, double2>::type;
    real* sw = reinterpret_cast<real*>(smem_raw);                  // CH * 3 * PP
    real* sc = sw + CH * 3 * PP;                                   // P * (degw + 1)
    real* srho = sc + P * (degw + 1);                              // CH
    int* soff = reinterpret_cast<int*>(srho + CH);                 // CH
    for (int i = threadIdx.x; i < P * (degw + 1); i += blockDim.x) sc[i] = wcoef[i];

    const int col = threadIdx.x;
    const bool own = col < E * E;
    const int b = col / E, c = col % E;
    real acc[E];
#pragma unroll
    for (int a = 0; a < E; ++a) acc[a] = real(0);
    real* heads = scratch;
    real* tails = scratch + static_cast<size_t>(ch.ntiles) * T * E * E;

    for (int k = 0; k < ch.K; ++k) {
    const int tile = (qx * ch.K + k) * ch.nyz + rem;
    const int beg = tile_off[tile], end = tile_off[tile + 1];
    for (int base = beg; base < end; base += CH) {
        const int cnt = min(CH, end - base);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * 3; t += blockDim.x) {
            const int j = t / 3, d = t % 3;
            const Vec4<real> r = rec[base + j];
            const real z = d == 0 ? r.x : (d == 1 ? r.y : r.z);
            real w[P];
            window_weights<real, P>(sc, degw, z, w);
#pragma unroll
            for (int a = 0; a < P; ++a) sw[(j * 3 + d) * PP + a] = w[a];
            if (d == 0) {
                srho[j] = r.w;
                soff[j] = idx[base + j].x;
            }
        }
        __syncthreads();
        if (own) {
            for (int j = 0; j < cnt; ++j) {
                const int pk = soff[j];
                const int ox = pk & 0xff, oy = (pk >> 8) & 0xff, oz = (pk >> 16) & 0xff;
                const int bb = b - oy, cc = c - oz;
                if (bb < 0 || bb >= P || cc < 0 || cc >= P) continue;
                const real wyz = srho[j] * sw[(j * 3 + 1) * PP + bb] * sw[(j * 3 + 2) * PP + cc];
                real wx[PP];
                const V* wv = reinterpret_cast<const V*>(sw + (j * 3) * PP);
#pragma unroll
                for (int v = 0; v < PP / VW; ++v) {
                    const V t = wv[v];
                    if constexpr (sizeof(real) == 4) {
                        wx[4 * v] = t.x;
                        wx[4 * v + 1] = t.y;
                        wx[4 * v + 2] = t.z;
                        wx[4 * v + 3] = t.w;
                    } else {
                        wx[2 * v] = t.x;
                        wx[2 * v + 1] = t.y;
                    }
                }
                switch (ox) {
#define PSWF_SPREAD_CASE(O)                                                                    \
    case O:                                                                                    \
        if constexpr (O < T) {                                                                 \
            _Pragma("unroll") for (int p = 0; p < P; ++p) acc[O + p] = fma(wyz, wx[p], acc[O + p]); \
        }                                                                                      \
        break;
                    PSWF_SPREAD_CASE(0)
                    PSWF_SPREAD_CASE(1)
                    PSWF_SPREAD_CASE(2)
                    PSWF_SPREAD_CASE(3)
                    PSWF_SPREAD_CASE(4)
                    PSWF_SPREAD_CASE(5)
                    PSWF_SPREAD_CASE(6)
                    PSWF_SPREAD_CASE(7)
#undef PSWF_SPREAD_CASE
                    default: break;
                }
            }
        }
    }
    // planes [0, T) of this tile are complete along x within the chain (later tiles start T further):
    // write them as the tile's head and carry the remaining E - T planes to the next tile
    if (own) {
        real* out = heads + static_cast<size_t>(tile) * T * E * E;
#pragma unroll
        for (int a = 0; a < T; ++a) out[a * E * E + col] = acc[a];
#pragma unroll
        for (int a = 0; a < E; ++a) acc[a] = a + T < E ? acc[a + T] : real(0);
    }
    }
    if (own) {   // the chain's tail: planes that belong to the tiles after the chain
        real* out = tails + static_cast<size_t>(bx) * (E - T) * E * E;
#pragma unroll
        for (int a = 0; a < E - T; ++a) out[a * E * E + col] = acc[a];
    }
}

template <typename real, int P>
__global__ void __launch_bounds__(spread_threads<P, spread_tile<real>()>()) k_spread(const Vec4<real>* __restrict__ rec, const int2* __restrict__ idx,
                                                 const int* __restrict__ tile_off, const real* __restrict__ wcoef,
                                                 int degw, SpreadChain ch, real* __restrict__ scratch) {
    k_spread_body<real, P>(blockIdx.x, rec, idx, tile_off, wcoef, degw, ch, scratch);
}

// ---- Alg. 2 step 1 (continued): halo sum of the tile slabs into the periodic grid -----------------
// Grid point l gets, from every tile column (t_y, t_z) overlapping it in y and z (ceil(E / T) per axis,
// periodic), the head of its own x tile at plane l_x mod T and the tails of the x-chains that end
// before l_x and still reach it (at most one unless the chain is shorter than E - T).  Every slab value
// is read by exactly one grid point per overlapping column.  NI > 0 (float32 plans, tile edge 8 at
// compile time, NI = ceil(E / T)): the y-z enumeration is unrolled, blocks of 32 x 8 points (z, y) and
// grid (m_z / 32, m_y / 8, m_x).  NI = 0: run-time tile edge, one thread per point of a 1-D grid.
template <typename real, int NI>
__device__ __forceinline__ void k_halo_body(int bx, int by, const real* __restrict__ scratch, const int* __restrict__ tile_off,
                                            Geom g, real* __restrict__ grid) {
    (void)tile_off;
    const int my = g.m[1], mz = g.m[2], P = g.P;
    const int nty = g.nt[1], ntz = g.nt[2], K = g.K, nchx = g.nt[0] / g.K;
    const int T = NI > 0 ? kTile32 : g.T, E = T + P - 1, ET = E - T;
    const size_t plane = static_cast<size_t>(E) * E;
    const real* heads = scratch;
    const real* tails = scratch + static_cast<size_t>(g.nt[0]) * nty * ntz * T * plane;
    int lx, ly, lz;
    if constexpr (NI > 0) {   // 32 x 8 blocks over (z, y), blockIdx.z = x
        lz = bx * 32 + static_cast<int>(threadIdx.x);
        ly = by * 8 + static_cast<int>(threadIdx.y);
        lx = blockIdx.z;
        if (lz >= mz || ly >= my) return;
    } else {
        const int id = bx * blockDim.x + threadIdx.x;
        if (id >= g.m[0] * my * mz) return;
        lz = id % mz;
        ly = (id / mz) % my;
        lx = id / (mz * my);
    }
    const int tlx = lx / T, tly = ly / T, tlz = lz / T;
    const int olx = lx - tlx * T, oly = ly - tly * T, olz = lz - tlz * T;
    const int qc = tlx / K;   // the chain holding lx; the tails of the chains before it reach into lx
    real s = real(0);
    auto add_column = [&](int tyz, int ey, int ez) {
        s += heads[(static_cast<size_t>(tlx) * nty * ntz + tyz) * T * plane + olx * plane + ey * E + ez];
        for (int j = 1;; ++j) {
            const int e = lx - (qc - j + 1) * K * T;   // plane of chain qc - j's tail at lx
            if (e >= ET) break;
            int q = (qc - j) % nchx;
            q += q < 0 ? nchx : 0;
            s += tails[(static_cast<size_t>(q) * nty * ntz + tyz) * ET * plane + e * plane + ey * E + ez];
        }
    };
    if constexpr (NI > 0) {
        int tys[NI], tzs[NI];
#pragma unroll
        for (int a = 0; a < NI; ++a) {   // tiny grids wrap repeatedly
            int t = tly - a;
            while (t < 0) t += nty;
            tys[a] = t;
            t = tlz - a;
            while (t < 0) t += ntz;
            tzs[a] = t;
        }
#pragma unroll
        for (int b = 0; b < NI; ++b) {
            const int ey = oly + b * T;
#pragma unroll
            for (int c = 0; c < NI; ++c) {
                const int ez = olz + c * T;
                if (ey < E && ez < E) add_column(tys[b] * ntz + tzs[c], ey, ez);
            }
        }
        grid[(static_cast<size_t>(lx) * my + ly) * mz + lz] = s;
    } else {
        int ty = tly;
        for (int ey = oly; ey < E; ey += T) {
            int tz = tlz;
            for (int ez = olz; ez < E; ez += T) {
                add_column(ty * ntz + tz, ey, ez);
                tz = tz == 0 ? ntz - 1 : tz - 1;
            }
            ty = ty == 0 ? nty - 1 : ty - 1;
        }
        grid[(static_cast<size_t>(lx) * my + ly) * mz + lz] = s;
    }
}

template <typename real, int NI>
__global__ void __launch_bounds__(256) k_halo(const real* __restrict__ scratch, const int* __restrict__ tile_off, Geom g,
                                              real* __restrict__ grid) {
    k_halo_body<real, NI>(blockIdx.x, blockIdx.y, scratch, tile_off, g, grid);
}

// ---- Alg. 2 step 3: diagonal scaling on the R2C half spectrum ------------------------------------
// Cube: S = mtab[|k|^2] iw[kx] iw[ky] iw[kz] on the open ball |k| < m/2 (host table over integer |k|^2).
// Cuboid: |omega|^2 = sum_d (2 pi k_d / L_d)^2 is not an integer function, so
// S = (4 pi / (V |omega|^2)) g(2 t - 1) iw_x[kx] iw_y[ky] iw_z[kz] with t = (|omega| r_c / c_s)^2 < 1 (the
// retained ellipsoid) and g the host fit of the in-band mollifier transform psi(sqrt t)/psi(0).
template <typename real>
struct ScaleParams {
    int m[3];
    int cube, degg;
    real w2[3];          // (2 pi / L_d)^2
    real tscale;         // (r_c / c_s)^2
    real four_pi_over_V;
    const real* iw;      // cube: m entries; cuboid: m_x + m_y + m_z entries
    const real* mtab;    // cube only
    const real* gc;      // cuboid only: degg + 1 monomial coefficients
};

template <typename real, typename cplx>
__device__ __forceinline__ void k_scale_body(int bx, cplx* __restrict__ spec, ScaleParams<real> sp) {
    const int mx = sp.m[0], my = sp.m[1], mz = sp.m[2], mh = mz / 2 + 1;
    const int id = bx * blockDim.x + threadIdx.x;
    if (id >= mx * my * mh) return;
    const int iz = id % mh, iy = (id / mh) % my, ix = id / (mh * my);
    const int kx = ix < mx / 2 ? ix : ix - mx, ky = iy < my / 2 ? iy : iy - my, kz = iz;
    real s = real(0);
    if (sp.cube) {
        const int m = mx;
        const int q = kx * kx + ky * ky + kz * kz;
        const int qmax = (m / 2) * (m / 2);
        if (q > 0 && q < qmax) s = sp.mtab[q] * sp.iw[ix] * sp.iw[iy] * sp.iw[iz];   // open ball |k| < m/2
    } else {
        const real w2 = sp.w2[0] * real(kx * kx) + sp.w2[1] * real(ky * ky) + sp.w2[2] * real(kz * kz);
        const real t = w2 * sp.tscale;
        if (w2 > real(0) && t < real(1)) {
            const real u = real(2) * t - real(1);
            real gh = sp.gc[sp.degg];
            for (int k = sp.degg - 1; k >= 0; --k) gh = fma(gh, u, sp.gc[k]);
            s = sp.four_pi_over_V / w2 * gh * sp.iw[ix] * sp.iw[mx + iy] * sp.iw[mx + my + iz];
        }
    }
    cplx v = spec[id];
    v.x *= s;
    v.y *= s;
    spec[id] = v;
}

template <typename real, typename cplx>
__global__ void k_scale(cplx* __restrict__ spec, ScaleParams<real> sp) {
    k_scale_body<real, cplx>(blockIdx.x, spec, sp);
}

// ---- Alg. 2 step 5 with eq. force: interpolation of phi and grad phi ------------------------------
// One CTA per tile: the tile's extended block of the grid b (E^3 values) is staged in shared memory.
// Each warp takes batches of NB particles: all 32 lanes first evaluate the 6 P window weights
// (value and x-derivative per axis) of the batch, one (particle, axis, kind) Horner vector per lane,
// then contract each particle's P^3 stencil cooperatively: lanes take (b, c) pairs, reduce over a in
// registers (two independent chains), and the warp sums the four results with shuffles.
// The block is stored y-major ([y][x][z]) with the y-plane stride padded to SP = P (mod 32): lane
// q = b P + c of a particle then reads word q (mod 32) of its x-row, so the 32 lanes hit 32 different
// banks (a z-row-major block of width E = T + P - 1 put two y-rows on the same banks).
template <int P, int E>
constexpr int interp_plane() { return E * E + (((P - E * E) % 32) + 32) % 32; }
template <typename real> struct InterpCfg;
template <> struct InterpCfg<float> { static constexpr int NB = 8, NWARP = 8; };
template <> struct InterpCfg<double> { static constexpr int NB = 8, NWARP = 4; };

// Stages the tile's extended block of the grid, x in [tx T, tx T + E) (and y, z alike, periodic), as
// G[y SP + x E + z].  The block's E^2 z-rows are contiguous in the grid unless they cross the periodic
// end, and every row starts on a 16-byte boundary (z0 = tz T, T multiple of 16 / sizeof(real), m_z a
// multiple of T, the grid 256-byte aligned): NV lanes load one row in 16-byte vectors (the last vector
// may read up to VW - 1 values past the row, still inside the grid), 32 / NV rows per warp step.  Tiles
// whose rows wrap (the last ones along z, or E > m) load element by element.
template <typename real, int T, int E, int SP, int NWARP>
__device__ __forceinline__ void stage_block(const real* __restrict__ grid, int mx, int my, int mz, int tx, int ty,
                                            int tz, int lane, int warp, real* __restrict__ G) {
    constexpr int VW = 16 / static_cast<int>(sizeof(real)), NV = (E + VW - 1) / VW, RPW = 32 / NV;
    using V = typename std::conditional<sizeof(real) == 4, float4, double2>::type;
    static_assert((T * sizeof(real)) % 16 == 0, "tile rows must start on 16-byte boundaries");
    auto wrap = [](int v, int m) {
        while (v >= m) v -= m;   // v < 2 m except for blocks wider than the grid
        return v;
    };
    const int z0 = tz * T;
    if (z0 + NV * VW <= mz && E <= mx && E <= my) {
        const int rl = lane / NV, k = lane - rl * NV;   // row of the warp step, vector in the row
        for (int r0 = warp * RPW; r0 < E * E; r0 += NWARP * RPW) {
            const int row = r0 + rl;
            if (rl < RPW && row < E * E) {
                const int ex = row / E, ey = row - ex * E;
                const int gx = wrap(tx * T + ex, mx), gy = wrap(ty * T + ey, my);
                const V v = reinterpret_cast<const V*>(grid + (static_cast<size_t>(gx) * my + gy) * mz + z0)[k];
                real* dst = G + ey * SP + ex * E + k * VW;
                if constexpr (sizeof(real) == 4) {
                    dst[0] = v.x;
                    if (k * VW + 1 < E) dst[1] = v.y;
                    if (k * VW + 2 < E) dst[2] = v.z;
                    if (k * VW + 3 < E) dst[3] = v.w;
                } else {
                    dst[0] = v.x;
                    if (k * VW + 1 < E) dst[1] = v.y;
                }
            }
        }
    } else {
        for (int e = warp * 32 + lane; e < E * E * E; e += NWARP * 32) {
            const int ez = e % E, ey = (e / E) % E, ex = e / (E * E);
            const int gx = wrap(tx * T + ex, mx), gy = wrap(ty * T + ey, my), gz = wrap(z0 + ez, mz);
            G[ey * SP + ex * E + ez] = grid[(static_cast<size_t>(gx) * my + gy) * mz + gz];
        }
    }
}

template <typename real, int P>
__device__ __forceinline__ void k_interp_body(int bx, const real* __restrict__ grid, const Vec4<real>* __restrict__ rec,
                                                const int2* __restrict__ idx, const int* __restrict__ tile_off,
                                                const real* __restrict__ wcoef, const real* __restrict__ dwcoef,
                                                Geom g, Vec4<real> inv_alpha, double* __restrict__ phi_out,
                                                double* __restrict__ f_out) {
    constexpr int T = spread_tile<real>(), E = T + P - 1;
    constexpr int NB = InterpCfg<real>::NB, NWARP = InterpCfg<real>::NWARP;
    constexpr int NQ = (P * P + 31) / 32;
    const int tile = bx;
    const int beg = tile_off[tile], end = tile_off[tile + 1];
    if (beg == end) return;
    const int mx = g.m[0], my = g.m[1], mz = g.m[2], degw = g.degw;
    const int tz = tile % g.nt[2], ty = (tile / g.nt[2]) % g.nt[1], tx = tile / (g.nt[2] * g.nt[1]);
    // weight rows padded to whole 16-byte vectors (vector loads of a particle's x-weights)
    constexpr int VW = 16 / static_cast<int>(sizeof(real)), PP = (P + VW - 1) / VW * VW;
    using V = typename std::conditional<sizeof(real) == 4, float4, double2>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* sw = reinterpret_cast<real*>(smem_raw);                 // NWARP * NB * 6 * PP
    constexpr int SP = interp_plane<P, E>();
    real* G = sw + NWARP * NB * 6 * PP;                           // E planes of SP (y-major)
    // window and derivative coefficients by power, rows of PP (window_weights_rows)
    real* sc = G + (E * SP + VW - 1) / VW * VW;                   // (degw + 1) * PP
    real* sd = sc + PP * (degw + 1);                              // (degw + 1) * PP
    for (int i = threadIdx.x; i < PP * (degw + 1); i += blockDim.x) {
        const int k = i / PP, a = i - k * PP;
        sc[i] = a < P ? wcoef[a * (degw + 1) + k] : real(0);
        sd[i] = a < P ? dwcoef[a * (degw + 1) + k] : real(0);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    stage_block<real, T, E, SP, NWARP>(grid, mx, my, mz, tx, ty, tz, lane, warp, G);
    __syncthreads();
    real* ww = sw + warp * NB * 6 * PP;
    for (int b0 = beg + warp * NB; b0 < end; b0 += NWARP * NB) {
        const int cnt = min(NB, end - b0);
        __syncwarp();
        for (int task = lane; task < cnt * 6; task += 32) {
            const int j = task / 6, kind = task % 6, d = kind % 3;
            const Vec4<real> r = rec[b0 + j];
            const real z = d == 0 ? r.x : (d == 1 ? r.y : r.z);
            // kinds 0-2 are w_d, kinds 3-5 are w'_d / alpha_d.  The lanes of a warp hold mixed kinds, so
            // the coefficient rows and the factor are selected, not branched on (a branch would run both
            // Horner sums on half the lanes each); w x 1 is exact.
            const bool deriv = kind >= 3;
            const real s = deriv ? (d == 0 ? inv_alpha.x : (d == 1 ? inv_alpha.y : inv_alpha.z)) : real(1);
            real w[P];
            window_weights_rows<real, P, PP>(deriv ? sd : sc, degw, z, w);
            V* out = reinterpret_cast<V*>(ww + (j * 6 + kind) * PP);
#pragma unroll
            for (int v = 0; v < PP / VW; ++v) {
                real t[VW];
#pragma unroll
                for (int u = 0; u < VW; ++u) t[u] = VW * v + u < P ? w[VW * v + u] * s : real(0);
                if constexpr (sizeof(real) == 4) {
                    out[v] = make_float4(t[0], t[1], t[2], t[3]);
                } else {
                    out[v] = make_double2(t[0], t[1]);
                }
            }
        }
        __syncwarp();
        real mph = 0, mgx = 0, mgy = 0, mgz = 0;   // lane j keeps particle j's results
        for (int j = 0; j < cnt; ++j) {
            const int2 id = idx[b0 + j];
            const int ox = id.x & 0xff, oy = (id.x >> 8) & 0xff, oz = (id.x >> 16) & 0xff;
            const real* wp = ww + j * 6 * PP;
            real wx[PP], dwx[PP];
            {
                const V* v0 = reinterpret_cast<const V*>(wp);
                const V* v3 = reinterpret_cast<const V*>(wp + 3 * PP);
#pragma unroll
                for (int v = 0; v < PP / VW; ++v) {
                    const V a0 = v0[v], a3 = v3[v];
                    if constexpr (sizeof(real) == 4) {
                        wx[4 * v] = a0.x; wx[4 * v + 1] = a0.y; wx[4 * v + 2] = a0.z; wx[4 * v + 3] = a0.w;
                        dwx[4 * v] = a3.x; dwx[4 * v + 1] = a3.y; dwx[4 * v + 2] = a3.z; dwx[4 * v + 3] = a3.w;
                    } else {
                        wx[2 * v] = a0.x; wx[2 * v + 1] = a0.y;
                        dwx[2 * v] = a3.x; dwx[2 * v + 1] = a3.y;
                    }
                }
            }
            real ph = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll
            for (int qi = 0; qi < NQ; ++qi) {
                const int q = lane + 32 * qi;
                if (q < P * P) {
                    const int bb = q / P, cc = q - (q / P) * P;
                    const real* col = G + (oy + bb) * SP + ox * E + oz + cc;
                    real s1a = 0, s1b = 0, s2a = 0, s2b = 0;
#pragma unroll
                    for (int a = 0; a < P; a += 2) {
                        const real v = col[a * E];
                        s1a = fma(v, wx[a], s1a);
                        s2a = fma(v, dwx[a], s2a);
                        if (a + 1 < P) {
                            const real v2 = col[(a + 1) * E];
                            s1b = fma(v2, wx[a + 1], s1b);
                            s2b = fma(v2, dwx[a + 1], s2b);
                        }
                    }
                    const real s1 = s1a + s1b, s2 = s2a + s2b;
                    const real wy = wp[PP + bb], wz = wp[2 * PP + cc];
                    const real dwy = wp[4 * PP + bb], dwz = wp[5 * PP + cc];
                    const real yz = wy * wz;
                    ph = fma(s1, yz, ph);
                    gx = fma(s2, yz, gx);
                    gy = fma(s1, dwy * wz, gy);
                    gz = fma(s1, wy * dwz, gz);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ph += __shfl_xor_sync(0xffffffffu, ph, o);
                gx += __shfl_xor_sync(0xffffffffu, gx, o);
                gy += __shfl_xor_sync(0xffffffffu, gy, o);
                gz += __shfl_xor_sync(0xffffffffu, gz, o);
            }
            if (lane == j) {
                mph = ph;
                mgx = gx;
                mgy = gy;
                mgz = gz;
            }
        }
        // float64 outputs written lane-parallel: one float64 instruction stream per batch, not per
        // particle (float64 issue is ~1/64 of float32 on this GPU)
        if (lane < cnt) {
            const int i = idx[b0 + lane].y;
            const double q = static_cast<double>(rec[b0 + lane].w);
            phi_out[i] = static_cast<double>(mph) - g.self * q;
            f_out[3 * static_cast<size_t>(i) + 0] = -q * static_cast<double>(mgx);
            f_out[3 * static_cast<size_t>(i) + 1] = -q * static_cast<double>(mgy);
            f_out[3 * static_cast<size_t>(i) + 2] = -q * static_cast<double>(mgz);
        }
    }
}

template <typename real, int P>
__global__ void __launch_bounds__(32 * InterpCfg<real>::NWARP) k_interp(const real* __restrict__ grid, const Vec4<real>* __restrict__ rec,
                                                const int2* __restrict__ idx, const int* __restrict__ tile_off,
                                                const real* __restrict__ wcoef, const real* __restrict__ dwcoef,
                                                Geom g, Vec4<real> inv_alpha, double* __restrict__ phi_out,
                                                double* __restrict__ f_out) {
    k_interp_body<real, P>(blockIdx.x, grid, rec, idx, tile_off, wcoef, dwcoef, g, inv_alpha, phi_out, f_out);
}

// ---- real-space sum of R over the cell list (Sec. 3.1.1) -----------------------------------------
// Real-space sum over a cell list of cells of edge >= rc/R along x and y and >= rc/Rz along z (Rz = R
// for float64 and float-float plans, 4 for float32 plans).  Cells are stored z-fastest, so a run of cells
// along z in one (x, y) column is one contiguous particle range, or several where the run wraps around
// the periodic box (every wrapped piece is a different periodic image).
//
// float64 / float-float plans (k_short_q, k_short_ff): one warp per target cell; the source cells within
// reach form columns (dx, dy) with a z-run dz in [-dzmax, dzmax] keeping the box distance below rc (host
// table); the warp flattens the ranges into one candidate stream, tests 32 candidates at a time against
// the cell's targets in float32 and queues passing pairs for full-warp evaluation.
// float32 plans (k_short): one target at a time, over its own neighbourhood (target_ranges).
// Pairs are evaluated in the plan's precision:
//   R(r) = 1/r - P1(u),  -R'(r)/r = 1/r^3 + Q(u),  u = 2 r^2/rc^2 - 1   (host-fitted polynomials).
// In float32 the displacement is float-float: positions are (hi, lo) pairs relative to their cell and
// the cell shift d w is split the same way, d = (hi_i - (hi_j + s_hi)) + ((lo_i - s_lo) - lo_j), so a
// close pair across a cell face keeps full relative precision.  In float64, 1/r is the float32
// reciprocal square root refined by two Newton steps y <- y (3 - r^2 y^2) / 2.
template <typename real>
__device__ __forceinline__ real rsqrt_r(real v);
template <> __device__ __forceinline__ float rsqrt_r<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_r<double>(double v) {
    double y = static_cast<double>(rsqrtf(static_cast<float>(v)));
    const double hv = 0.5 * v;
    y = y * fma(-hv * y, y, 1.5);
    y = y * fma(-hv * y, y, 1.5);
    return y;
}

constexpr int kShortWarps = 4;      // target cells per block
constexpr int kShortMaxT = 8;       // targets per pass
constexpr int kShortMaxR = 4;       // largest reach
constexpr int kShortMaxRanges = 256;   // >= 81 columns x 3 pieces (nc >= 2R since rc <= L/2)

// Per-warp range arrays of the real-space kernels live in dynamic shared memory, sized by the host's
// bound on the pieces of one neighbourhood (columns x pieces per column <= kShortMaxRanges).
__host__ __device__ constexpr size_t short_dyn_smem(int rcap) {
    return static_cast<size_t>(kShortWarps) * (16u * rcap + 4u * (rcap + 1));
}
// float32 kernel (k_short): the ranges, their x-y cell shifts (float4 per piece) and the offsets
__host__ __device__ constexpr size_t short_dyn_smem_f32(int rcap) {
    return static_cast<size_t>(kShortWarps) * (32u * rcap + 4u * (rcap + 1));
}

// Flattens the source ranges of target cell (cx, cy, cz) for one warp: every column (dx, dy, dzmax) of
// scol contributes its z-run dz in [-dzmax, dzmax], split into contiguous pieces of the z-fastest cell
// order (one piece per wrap of the periodic box).  rng[r] = {first particle, first z cell, dz of that
// cell, column}, pos[r] = offset of piece r in the flattened candidate stream, pos[nr] = total.
// Returns the total number of candidates (warp-uniform).  Pieces beyond cap are dropped; the host sizes
// cap from the columns and the largest number of pieces per column, so none are.
__device__ __forceinline__ int short_ranges(const int4* __restrict__ scol, int ncols, const int* __restrict__ cell_off,
                                            const int* nc3, int cx, int cy, int cz, int lane, int cap, int4* rng,
                                            int* pos) {
    const int ncx = nc3[0], ncy = nc3[1], nc = nc3[2];   // nc: cells along z (the contiguous axis)
    auto wrapn = [](int v, int n) {   // v in (-2 n, 2 n) -> [0, n)
        v += v < 0 ? n : 0;
        v += v < 0 ? n : 0;
        v -= v >= n ? n : 0;
        v -= v >= n ? n : 0;
        return v;
    };
    auto wrap = [&](int v) { return wrapn(v, nc); };
    int nr = 0;
    for (int k0 = 0; k0 < ncols; k0 += 32) {
        const int k = k0 + lane;
        int npc = 0;
        int4 col = make_int4(0, 0, -1, 0);
        int base = 0;
        if (k < ncols) {
            col = scol[k];
            base = (wrapn(cx + col.x, ncx) * ncy + wrapn(cy + col.y, ncy)) * nc;
            for (int d = -col.z; d <= col.z;) {
                const int zw = wrap(cz + d);
                d += min(col.z - d + 1, nc - zw);
                ++npc;
            }
        }
        int incl = npc;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int slot = nr + incl - npc;
        if (k < ncols) {
            for (int d = -col.z; d <= col.z;) {
                const int zw = wrap(cz + d);
                const int len = min(col.z - d + 1, nc - zw);
                if (slot < cap) {
                    const int a = cell_off[base + zw], b = cell_off[base + zw + len];
                    rng[slot] = make_int4(a, zw, d, k);
                    pos[slot] = b - a;            // length, turned into offsets below
                }
                ++slot;
                d += len;
            }
        }
        nr += __shfl_sync(0xffffffffu, incl, 31);
    }
    nr = min(nr, cap);
    __syncwarp();
    int total = 0;
    for (int r0 = 0; r0 < nr; r0 += 32) {
        const int r = r0 + lane;
        const int len = r < nr ? pos[r] : 0;
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __syncwarp();
        if (r < nr) pos[r] = total + incl - len;
        total += __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
    }
    if (lane == 0) pos[nr] = total;
    __syncwarp();
    return total;
}

// Per-target pair queues of the two-phase real-space kernels (k_short_q, k_short_ff).  The float32
// cutoff scan of a chunk of 32 candidates appends each passing (source, target t) pair to queue t
// (warp ballot + prefix popcount); every queue holding 32 or more pairs is drained by one full-warp
// evaluation with t warp-uniform, so the accumulation needs no per-lane target selection.
constexpr int kShortQCap = 64;   // < 32 left after a drain, at most 32 added per chunk

__device__ __forceinline__ void short_enqueue(unsigned mask, int nt, int2 entry, int lane, int2 (*queue)[kShortQCap],
                                              int* qlen) {
    const unsigned lt = (1u << lane) - 1u;
    for (int t = 0; t < nt; ++t) {
        const bool mine = (mask >> t) & 1u;
        const unsigned b = __ballot_sync(0xffffffffu, mine);
        if (mine) queue[t][qlen[t] + __popc(b & lt)] = entry;
        __syncwarp();
        if (lane == 0) qlen[t] += __popc(b);
        __syncwarp();
    }
}

// Per-plan constants of the real-space kernel, passed by value (kernel parameter space): the radial
// polynomials padded with leading zeros to the compile-time degree D, so the fully unrolled Horner
// loops read every coefficient as a constant operand.
template <typename real, int D>
struct ShortParams {
    real p1[D + 1], q[D + 1];
    real rc2, two_over_rc2;
    float rc2f;
};

// Source ranges of ONE target for the float32 real-space sum: every column (dx, dy) of the reach whose
// x-y box distance from the target point is below the cutoff contributes the run of z cells that can
// hold points within the cutoff of the target (its z window, from the target's own position), split
// into contiguous pieces at the periodic wrap.  Lanes take one column each.  rng[r] = {first particle,
// first z cell, dz of that cell, ix | iy << 4}, shf[r] = the piece's x and y cell shifts {hi x, hi y,
// lo x, lo y}, pos[r] = offset of piece r in the candidate stream, pos[nr] = total, returned
// (warp-uniform).  Columns whose pieces would overflow cap are dropped (the
// host sizes cap for the worst case, so none are).
// v in (-2 n, 2 n) -> [0, n): periodic cell index
__device__ __forceinline__ int wrap_cells(int v, int n) {
    v += v < 0 ? n : 0;
    v += v < 0 ? n : 0;
    v -= v >= n ? n : 0;
    v -= v >= n ? n : 0;
    return v;
}

struct CellGridF {   // what target_ranges needs of the cell grid, in registers
    int R, Rz, ncx, ncy, nc;   // reach along x, y and along z; cells per axis
    float wx, wy, iwz;
};

__device__ __forceinline__ int target_ranges(const int* __restrict__ cell_off, const CellGridF cg, int cx, int cy,
                                             int cz, float tx, float ty, float tz, float rc2f, int lane, int cap,
                                             int4* rng, int* pos, const float* __restrict__ shx_hi,
                                             const float* __restrict__ shy_hi, const float* __restrict__ shx_lo,
                                             const float* __restrict__ shy_lo, float4* shf) {
    const int R = cg.R, Rz = cg.Rz, W = 2 * R + 1;
    const int ncx = cg.ncx, ncy = cg.ncy, nc = cg.nc;
    const float wx = cg.wx, wy = cg.wy, iwz = cg.iwz;
    const int divW = (65536 + W - 1) / W;   // k / W = (k divW) >> 16 exactly for k < W^2 <= 81
    int nr = 0;
    for (int k0 = 0; k0 < W * W; k0 += 32) {
        const int k = k0 + lane;
        int npc = 0, zlo = 0, zhi = -1, base = 0, dx = 0, dy = 0;
        if (k < W * W) {
            const int qd = (k * divW) >> 16;
            dx = qd - R;
            dy = k - qd * W - R;
            const float gx = dx > 0 ? dx * wx - tx : (dx < 0 ? tx - (dx + 1) * wx : 0.f);
            const float gy = dy > 0 ? dy * wy - ty : (dy < 0 ? ty - (dy + 1) * wy : 0.f);
            const float d2 = gx * gx + gy * gy;
            if (d2 < rc2f) {
                const float hz = sqrtf(rc2f - d2);
                zlo = max(-Rz, static_cast<int>(floorf((tz - hz) * iwz)));
                zhi = min(Rz, static_cast<int>(floorf((tz + hz) * iwz)));
                base = (wrap_cells(cx + dx, ncx) * ncy + wrap_cells(cy + dy, ncy)) * nc;
                for (int d = zlo; d <= zhi;) {
                    const int zw = wrap_cells(cz + d, nc);
                    d += min(zhi - d + 1, nc - zw);
                    ++npc;
                }
            }
        }
        int incl = npc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int slot = nr + incl - npc;
        for (int d = zlo; d <= zhi;) {
            const int zw = wrap_cells(cz + d, nc);
            const int len = min(zhi - d + 1, nc - zw);
            if (slot < cap) {
                const int a = cell_off[base + zw], b = cell_off[base + zw + len];
                rng[slot] = make_int4(a, zw, d, (dx + R) | ((dy + R) << 4));
                shf[slot] = make_float4(shx_hi[dx + R], shy_hi[dy + R], shx_lo[dx + R], shy_lo[dy + R]);
                pos[slot] = b - a;
            }
            ++slot;
            d += len;
        }
        nr += __shfl_sync(0xffffffffu, incl, 31);
    }
    nr = min(nr, cap);
    __syncwarp();
    int total = 0;
    for (int r0 = 0; r0 < nr; r0 += 32) {
        const int r = r0 + lane;
        const int len = r < nr ? pos[r] : 0;
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __syncwarp();
        if (r < nr) pos[r] = total + incl - len;
        total += __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
    }
    if (lane == 0) pos[nr] = total;
    __syncwarp();
    return total;
}

// float32 plans.  Each warp takes kShortTPW consecutive targets (cell order) one at a time: the lanes
// first build the target's own neighbourhood (target_ranges: z windows per column from the target's
// position), then test 32 candidates at a time against the cutoff and push the pairs inside it onto a
// per-warp ring in shared memory (ballot + prefix count); whenever 32 pairs are queued, the warp
// evaluates them with every lane busy.  The radial polynomials thus run once per pair inside r_c
// (~28% of the candidates at the bench plan), never under a divergent branch.  One warp reduction per
// target.  Measured split at n = 1e5, m = 96 (one launch): neighbourhood construction ~30%, cutoff
// tests ~53%, queued pair evaluation ~17% of the time.
//   R(r) = 1/r - P1(u),  -R'(r)/r = 1/r^3 + Q(u),  u = 2 r^2/rc^2 - 1   (host-fitted polynomials)
// Displacements are float-float: positions are (hi, lo) pairs relative to their cell and the cell shift
// d w is split the same way, d = (hi_t - (hi_j + s_hi)) + ((lo_t - lo_j) - s_lo), so a close pair
// across a cell face keeps its relative precision.
constexpr int kShortTPW = 4;   // targets per warp
constexpr int kShortRing = 64;   // queued pairs per warp: < 32 left over + 32 from one pass

template <int D>
__device__ __forceinline__ void k_short_body(int bx, const Vec4<float>* __restrict__ rec, const int2* __restrict__ idx,
                                                            const Vec4<float>* __restrict__ lo,
                                                            const int* __restrict__ cell_off, int rcap, Geom g,
                                                            const ShortParams<float, D>& kp,
                                                            float* __restrict__ phi_out, float* __restrict__ f_out) {
    constexpr int NSH = 2 * kShortMaxR + 1;
    __shared__ float sh_hi[3][NSH], sh_lo[3][NSH];   // cell shifts (k - R) w_d, hi and lo parts
    __shared__ float4 sh_q[kShortWarps][kShortRing];   // queued pairs {dx, dy, dz, q_j}
    const int R = g.reach, Rz = g.reachz;
    for (int k = threadIdx.x; k < 3 * NSH; k += blockDim.x) {
        const int d = k / NSH, i = k % NSH, rd = d == 2 ? Rz : R;
        const double w = d == 0 ? g.cellw[0] : (d == 1 ? g.cellw[1] : g.cellw[2]);
        const double o = (i - rd) * w;
        sh_hi[d][i] = static_cast<float>(o);
        sh_lo[d][i] = static_cast<float>(o - static_cast<double>(sh_hi[d][i]));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;   // lanes under this one
    extern __shared__ __align__(16) unsigned char short_dyn[];
    int4* rng = reinterpret_cast<int4*>(short_dyn) + warp * rcap;
    float4* shf = reinterpret_cast<float4*>(short_dyn) + kShortWarps * rcap + warp * rcap;
    int* pos = reinterpret_cast<int*>(reinterpret_cast<float4*>(short_dyn) + 2 * kShortWarps * rcap) + warp * (rcap + 1);
    float4* ring = sh_q[warp];
    const int t0 = (bx * kShortWarps + warp) * kShortTPW;
    const CellGridF cg{R, Rz, g.ncell[0], g.ncell[1], g.ncell[2], static_cast<float>(g.cellw[0]),
                       static_cast<float>(g.cellw[1]), static_cast<float>(g.invcellw[2])};
    for (int ti = t0; ti < min(t0 + kShortTPW, g.n); ++ti) {
        const Vec4<float> th = rec[ti];                 // same address in every lane: one broadcast load
        const Vec4<float> tl = lo[ti];
        const int c = idx[ti].x;   // packed cell coordinates
        const int cx = c & 1023, cy = (c >> 10) & 1023, cz = c >> 20;
        const int total = target_ranges(cell_off, cg, cx, cy, cz, th.x, th.y, th.z, kp.rc2f, lane, rcap, rng, pos,
                                        sh_hi[0], sh_hi[1], sh_lo[0], sh_lo[1], shf);
        float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        // one queued pair per lane: ring[(head + lane) mod ring] for lanes below cnt, zeros elsewhere
        auto evaluate = [&](int head, int cnt) {
            __syncwarp();   // the queued pairs are visible to every lane
            const bool valid = lane < cnt;
            const float4 e = valid ? ring[(head + lane) & (kShortRing - 1)] : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();   // read before the next pass may overwrite the slots
            const float r2 = valid ? fmaf(e.x, e.x, fmaf(e.y, e.y, e.z * e.z)) : 1.f;
            const float u = fmaf(r2, kp.two_over_rc2, float(-1));
            float p1 = kp.p1[D], qq = kp.q[D];
#pragma unroll
            for (int kk = D - 1; kk >= 0; --kk) {
                p1 = fmaf(p1, u, kp.p1[kk]);
                qq = fmaf(qq, u, kp.q[kk]);
            }
            const float ri = rsqrtf(r2);
            const float cf = e.w * fmaf(ri * ri, ri, qq);
            ph = fmaf(e.w, ri - p1, ph);
            gx = fmaf(cf, e.x, gx);
            gy = fmaf(cf, e.y, gy);
            gz = fmaf(cf, e.z, gz);
        };
        int r = 0, head = 0, queued = 0;   // ring head and fill (warp-uniform)
        for (int s0 = 0; s0 < total; s0 += 32) {   // warp-uniform trip count
            const int p = s0 + lane;
            bool in = false;
            float ddx = 0.f, ddy = 0.f, ddz = 0.f, qj = 0.f;
            if (p < total) {
                while (pos[r + 1] <= p) ++r;
                const int4 rg = rng[r];
                const float4 sf = shf[r];   // the piece's x, y shifts (hi, lo)
                const int j = rg.x + (p - pos[r]);
                const Vec4<float> a = rec[j];
                const Vec4<float> l = lo[j];
                const int iz = rg.z + (__float_as_int(l.w) - rg.y) + Rz;
                ddx = (th.x - (a.x + sf.x)) + ((tl.x - l.x) - sf.z);
                ddy = (th.y - (a.y + sf.y)) + ((tl.y - l.y) - sf.w);
                ddz = (th.z - (a.z + sh_hi[2][iz])) + ((tl.z - l.z) - sh_lo[2][iz]);
                const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
                in = r2 < kp.rc2 && r2 > 0.f;
                qj = a.w;
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (in) ring[(head + queued + __popc(m & below)) & (kShortRing - 1)] = make_float4(ddx, ddy, ddz, qj);
            queued += __popc(m);
            if (queued >= 32) {   // a full warp of pairs: ring[head .. head + 31]
                evaluate(head, 32);
                head = (head + 32) & (kShortRing - 1);
                queued -= 32;
            }
        }
        if (queued > 0) evaluate(head, queued);
        __syncwarp();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ph += __shfl_xor_sync(0xffffffffu, ph, o);
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
        }
        if (lane == 0) {   // float32 results; k_combine_energy widens them with full warps
            const int oi = idx[ti].y;
            phi_out[oi] = ph;
            f_out[3 * static_cast<size_t>(oi) + 0] = th.w * gx;
            f_out[3 * static_cast<size_t>(oi) + 1] = th.w * gy;
            f_out[3 * static_cast<size_t>(oi) + 2] = th.w * gz;
        }
        __syncwarp();
    }
}

template <int D>
__global__ void __launch_bounds__(32 * kShortWarps) k_short(const Vec4<float>* __restrict__ rec, const int2* __restrict__ idx,
                                                            const Vec4<float>* __restrict__ lo,
                                                            const int* __restrict__ cell_off, int rcap, Geom g,
                                                            const __grid_constant__ ShortParams<float, D> kp,
                                                            float* __restrict__ phi_out, float* __restrict__ f_out) {
    k_short_body<D>(blockIdx.x, rec, idx, lo, cell_off, rcap, g, kp, phi_out, f_out);
}

// Two-phase form of k_short (float64 plans): the float32 cutoff scan fills per-target pair queues, full
// warps of queued pairs are evaluated with the arithmetic of k_short, so the costly float64 pair
// evaluation runs without divergence.
template <int D>
__global__ void __launch_bounds__(32 * kShortWarps) k_short_q(const Vec4<double>* __restrict__ rec, const int2* __restrict__ idx,
                                                              const float4* __restrict__ pf,
                                                              const int* __restrict__ cell_off, const int4* __restrict__ cols,
                                                              int ncols, int rcap, Geom g, const __grid_constant__ ShortParams<double, D> kp,
                                                              double* __restrict__ phi_out, double* __restrict__ f_out) {
    constexpr int NSH = 2 * kShortMaxR + 1, MT = kShortMaxT;
    static_assert(NSH <= 16, "queue entries pack 4-bit shift indices");
    __shared__ float sh_hi[3][NSH];
    __shared__ double sh_d[3][NSH];
    __shared__ int4 scol[(2 * kShortMaxR + 1) * (2 * kShortMaxR + 1)];
    __shared__ double stx[kShortWarps][MT][4];          // exact target position and charge
    __shared__ float stl[kShortWarps][MT][4];         // float32 copy of the target (cutoff pre-test)
    __shared__ int2 sq[kShortWarps][MT][kShortQCap];  // {source, ix | iy << 4 | iz << 8}
    __shared__ int sqlen[kShortWarps][MT];
    const int R = g.reach, Rz = g.reachz;
    for (int k = threadIdx.x; k < 3 * NSH; k += blockDim.x) {
        const int d = k / NSH, i = k % NSH, rd = d == 2 ? Rz : R;
        const double o = (i - rd) * g.cellw[d];
        sh_d[d][i] = o;
        sh_hi[d][i] = static_cast<float>(o);
    }
    for (int k = threadIdx.x; k < ncols; k += blockDim.x) scol[k] = cols[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * kShortWarps + warp;
    if (c >= g.ncell[0] * g.ncell[1] * g.ncell[2]) return;
    const int tb = cell_off[c], te = cell_off[c + 1];
    if (tb == te) return;
    const int cz = c % g.ncell[2], cy = (c / g.ncell[2]) % g.ncell[1], cx = c / (g.ncell[2] * g.ncell[1]);
    extern __shared__ __align__(16) unsigned char short_dyn[];
    int4* rng = reinterpret_cast<int4*>(short_dyn) + warp * rcap;
    int* pos = reinterpret_cast<int*>(reinterpret_cast<int4*>(short_dyn) + kShortWarps * rcap) + warp * (rcap + 1);
    int* qlen = sqlen[warp];
    const int total = short_ranges(scol, ncols, cell_off, g.ncell, cx, cy, cz, lane, rcap, rng, pos);

    for (int t0 = tb; t0 < te; t0 += MT) {
        const int nt = min(MT, te - t0);
        __syncwarp();
        if (lane < nt) {
            const Vec4<double> a = rec[t0 + lane];
            stx[warp][lane][0] = a.x;
            stx[warp][lane][1] = a.y;
            stx[warp][lane][2] = a.z;
            stx[warp][lane][3] = a.w;
            const float4 f = pf[t0 + lane];
            stl[warp][lane][0] = f.x;
            stl[warp][lane][1] = f.y;
            stl[warp][lane][2] = f.z;
        }
        if (lane < MT) qlen[lane] = 0;
        __syncwarp();
        double acc[MT][4];
#pragma unroll
        for (int t = 0; t < MT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0;

        // evaluates one queued pair for target t (warp-uniform) and accumulates it
        auto pair = [&](int2 e, int t, bool active) {
            const int ix = e.y & 15, iy = (e.y >> 4) & 15, iz = (e.y >> 8) & 15;
            const Vec4<double> a = rec[active ? e.x : t0];
            double ddx, ddy, ddz;
            ddx = stx[warp][t][0] - (a.x + sh_d[0][ix]);
            ddy = stx[warp][t][1] - (a.y + sh_d[1][iy]);
            ddz = stx[warp][t][2] - (a.z + sh_d[2][iz]);
            const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            const bool in = active && r2 < kp.rc2 && r2 > 0.0;
            const double u = fma(r2, kp.two_over_rc2, double(-1));
            double p1 = kp.p1[D], qq = kp.q[D];
#pragma unroll
            for (int kk = D - 1; kk >= 0; --kk) {
                p1 = fma(p1, u, kp.p1[kk]);
                qq = fma(qq, u, kp.q[kk]);
            }
            const double ri = rsqrt_r<double>(in ? r2 : double(1));
            const double qj = in ? a.w : 0.0;
            const double c0 = qj * (ri - p1);
            const double cf = qj * fma(ri * ri, ri, qq);
#pragma unroll
            for (int tt = 0; tt < MT; ++tt)
                if (tt == t) {   // warp-uniform
                    acc[tt][0] += c0;
                    acc[tt][1] = fma(cf, ddx, acc[tt][1]);
                    acc[tt][2] = fma(cf, ddy, acc[tt][2]);
                    acc[tt][3] = fma(cf, ddz, acc[tt][3]);
                }
        };

        int r = 0;
        for (int s0 = 0;; s0 += 32) {   // one extra round after the last chunk flushes the queues
            const bool fin = s0 >= total;
            if (!fin) {
                // scan: float32 test of candidate p against every target of the pass
                const int p = s0 + lane;
                unsigned mask = 0u;
                int2 entry = make_int2(0, 0);
                if (p < total) {
                    while (pos[r + 1] <= p) ++r;
                    const int4 rg = rng[r];
                    const int j = rg.x + (p - pos[r]);
                    float sfx, sfy, sfz, szc;
                    const float4 f = pf[j];
                    sfx = f.x; sfy = f.y; sfz = f.z;
                    szc = f.w;
                    const int4 col = scol[rg.w];
                    const int ix = col.x + R, iy = col.y + R, iz = rg.z + (__float_as_int(szc) - rg.y) + Rz;
                    const float px = sfx + sh_hi[0][ix], py = sfy + sh_hi[1][iy], pz = sfz + sh_hi[2][iz];
#pragma unroll
                    for (int t = 0; t < MT; ++t) {
                        if (t >= nt) break;   // warp-uniform
                        float tx, ty, tz;
                        tx = stl[warp][t][0]; ty = stl[warp][t][1]; tz = stl[warp][t][2];
                        const float dxf = tx - px, dyf = ty - py, dzf = tz - pz;
                        const float r2f = dxf * dxf + dyf * dyf + dzf * dzf;
                        if (r2f < kp.rc2f && r2f > 0.f) mask |= 1u << t;
                    }
                    entry = make_int2(j, ix | (iy << 4) | (iz << 8));
                }
                short_enqueue(mask, nt, entry, lane, sq[warp], qlen);
            }
            // compute: drain every full queue (every non-empty one in the final round)
            for (int t = 0; t < nt; ++t) {
                while (qlen[t] >= 32 || (fin && qlen[t] > 0)) {
                    const int q = max(qlen[t] - 32, 0);
                    const bool act = lane < qlen[t] - q;
                    const int2 e = sq[warp][t][q + (act ? lane : 0)];
                    __syncwarp();
                    if (lane == 0) qlen[t] = q;
                    __syncwarp();
                    pair(e, t, act);
                }
            }
            if (fin) break;
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < MT; ++t) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                double x = acc[t][v];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                acc[t][v] = x;
            }
        }
        double mine[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            if (lane == t) {
                mine[0] = acc[t][0];
                mine[1] = acc[t][1];
                mine[2] = acc[t][2];
                mine[3] = acc[t][3];
            }
        }
        if (lane < nt) {
            const int oi = idx[t0 + lane].y;
            const double qi = static_cast<double>(stx[warp][lane][3]);
            phi_out[oi] = static_cast<double>(mine[0]);
            f_out[3 * static_cast<size_t>(oi) + 0] = qi * static_cast<double>(mine[1]);
            f_out[3 * static_cast<size_t>(oi) + 1] = qi * static_cast<double>(mine[2]);
            f_out[3 * static_cast<size_t>(oi) + 2] = qi * static_cast<double>(mine[3]);
        }
        __syncwarp();
    }
}

// ---- energy ------------------------------------------------------------------------------------
// phi += phi_sr, F += F_sr and E = 1/2 sum rho phi.  Block partial sums go to part[]; the last block to
// finish (ticket counter `done`, zeroed before the evaluation) adds them in a fixed order and writes E,
// so the energy needs no second launch and does not depend on the block schedule.  SR: the type of the
// real-space results (float for float32 plans: k_short leaves the widening to these full warps).
template <typename SR>
__device__ __forceinline__ void k_combine_energy_body(int bx, int nbx, double* __restrict__ phi, double* __restrict__ f,
                                                        const SR* __restrict__ phi_sr, const SR* __restrict__ f_sr,
                                                               const double* __restrict__ rho, int n,
                                                               double* __restrict__ part, unsigned* __restrict__ done,
                                                               double* __restrict__ energy) {
    double s = 0.0;
    for (int i = bx * blockDim.x + threadIdx.x; i < n; i += nbx * blockDim.x) {
        const double q = rho[i];
        const double p = phi[i] + static_cast<double>(phi_sr[i]);
        phi[i] = p;
        f[3 * static_cast<size_t>(i) + 0] += static_cast<double>(f_sr[3 * static_cast<size_t>(i) + 0]);
        f[3 * static_cast<size_t>(i) + 1] += static_cast<double>(f_sr[3 * static_cast<size_t>(i) + 1]);
        f[3 * static_cast<size_t>(i) + 2] += static_cast<double>(f_sr[3 * static_cast<size_t>(i) + 2]);
        s += ((__double2hiint(q) & 0x7ff00000) != 0x7ff00000 ? q : 0.0) * p;
    }
    __shared__ double red[8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[bx] = t;
        __threadfence();
        last = atomicAdd(done, 1u) == nbx - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < nbx; b += blockDim.x) t += __ldcg(part + b);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __syncthreads();
    if (lane == 0) red[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int w = 0; w < 8; ++w) e += red[w];
        energy[0] = 0.5 * e;
    }
}

template <typename SR>
__global__ void __launch_bounds__(256) k_combine_energy(double* __restrict__ phi, double* __restrict__ f,
                                                        const SR* __restrict__ phi_sr, const SR* __restrict__ f_sr,
                                                               const double* __restrict__ rho, int n,
                                                               double* __restrict__ part, unsigned* __restrict__ done,
                                                               double* __restrict__ energy) {
    k_combine_energy_body<SR>(blockIdx.x, gridDim.x, phi, f, phi_sr, f_sr, rho, n, part, done, energy);
}

}  // namespace pswf
