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
//   k_short    real-space sum of the residual R (eq. R) over the cell list, adds to phi, F
//   k_energy   E = 1/2 sum rho phi (Remark on energy), deterministic two-pass reduction
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pswf {

template <typename real> struct alignas(4 * sizeof(real)) Vec4 { real x, y, z, w; };

// Geometry and sizes shared by the kernels of one plan (passed by value).
struct Geom {
    int n, m, P, T, nt, ncell, reach, degw, degr;
    double L, invL, h, invh, cellw, rc, self;
};

constexpr int kTile = 4;   // spreading tile edge (grid points); m is a multiple of it

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
        double w = x - g.L * floor(x * g.invL);
        if (w >= g.L) w -= g.L;
        if (w < 0.0) w = 0.0;
        r.w[d] = w;
        const double t = w * g.invh;
        const int l0 = static_cast<int>(ceil(t - 0.5 * g.P));
        r.z[d] = 2.0 * (t - l0) - (g.P - 1);
        int lw = l0 % g.m;
        if (lw < 0) lw += g.m;
        r.lw[d] = lw;
        int c = static_cast<int>(w / g.cellw);
        c = c < 0 ? 0 : (c >= g.ncell ? g.ncell - 1 : c);
        r.cell[d] = c;
        r.loc[d] = w - c * g.cellw;
    }
    return r;
}

__device__ inline int tile_of(const Located& r, const Geom& g) {
    return ((r.lw[0] / g.T) * g.nt + r.lw[1] / g.T) * g.nt + r.lw[2] / g.T;
}
__device__ inline int cell_of(const Located& r, const Geom& g) {
    return (r.cell[0] * g.ncell + r.cell[1]) * g.ncell + r.cell[2];
}

// status[0] = sum rho, status[1] = sum |rho|, status[2] = number of non-finite inputs
static __global__ void k_prep(const double* __restrict__ x, const double* __restrict__ rho, Geom g,
                       int* __restrict__ key_rank, int* __restrict__ tile_cnt, int* __restrict__ cell_cnt,
                       double* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double q = 0.0, aq = 0.0, bad = 0.0;
    if (i < g.n) {
        const Located r = locate(x + 3 * static_cast<size_t>(i), g);
        double rq = rho[i];
        if (!isfinite(rq) || !r.finite) bad = 1.0;
        if (!isfinite(rq)) rq = 0.0;
        q = rq;
        aq = fabs(rq);
        const int t = tile_of(r, g), c = cell_of(r, g);
        const int rt = atomicAdd(tile_cnt + t, 1);
        const int rc = atomicAdd(cell_cnt + c, 1);
        int4 kr = make_int4(t, rt, c, rc);
        reinterpret_cast<int4*>(key_rank)[i] = kr;
    }
    // block reduction of the neutrality / finiteness diagnostics
    for (int o = 16; o > 0; o >>= 1) {
        q += __shfl_xor_sync(0xffffffffu, q, o);
        aq += __shfl_xor_sync(0xffffffffu, aq, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ double red[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = q; red[1][warp] = aq; red[2][warp] = bad; }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        q = lane < nw ? red[0][lane] : 0.0;
        aq = lane < nw ? red[1][lane] : 0.0;
        bad = lane < nw ? red[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            q += __shfl_xor_sync(0xffffffffu, q, o);
            aq += __shfl_xor_sync(0xffffffffu, aq, o);
            bad += __shfl_xor_sync(0xffffffffu, bad, o);
        }
        if (lane == 0) {
            atomicAdd(status + 0, q);
            atomicAdd(status + 1, aq);
            if (bad > 0) atomicAdd(status + 2, bad);
        }
    }
}

// Exclusive scan of cnt[0..N) into off[0..N]; one block per segment (blockIdx.x = 0 / 1).
static __global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ cnt0, int* __restrict__ off0, int n0,
                                               const int* __restrict__ cnt1, int* __restrict__ off1, int n1) {
    const int* cnt = blockIdx.x == 0 ? cnt0 : cnt1;
    int* off = blockIdx.x == 0 ? off0 : off1;
    const int N = blockIdx.x == 0 ? n0 : n1;
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int carry = 0;
    constexpr int ITEMS = 4;
    for (int base = 0; base < N; base += blockDim.x * ITEMS) {
        int v[ITEMS], s = 0;
        const int i0 = base + threadIdx.x * ITEMS;
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            v[k] = (i0 + k < N) ? cnt[i0 + k] : 0;
            s += v[k];
        }
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
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            if (i0 + k < N) off[i0 + k] = e;
            e += v[k];
        }
        const int total = wsum[nw - 1];
        __syncthreads();
        carry += total;
    }
    if (threadIdx.x == 0) off[N] = carry;
}

// Sorted records.  Spreading side (tile order): {z0, z1, z2, rho}, {packed offsets in tile, original index}.
// Real-space side (cell order): {local x, y, z, rho}, {cell id, original index}.
template <typename real>
__global__ void k_scatter(const double* __restrict__ x, const double* __restrict__ rho, Geom g,
                          const int* __restrict__ key_rank, const int* __restrict__ tile_off,
                          const int* __restrict__ cell_off, Vec4<real>* __restrict__ sp_rec,
                          int2* __restrict__ sp_idx, Vec4<real>* __restrict__ sr_rec, int2* __restrict__ sr_idx,
                          Vec4<real>* __restrict__ sr_lo) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const Located r = locate(x + 3 * static_cast<size_t>(i), g);
    double q = rho[i];
    if (!isfinite(q)) q = 0.0;
    const int4 kr = reinterpret_cast<const int4*>(key_rank)[i];
    const int ps = tile_off[kr.x] + kr.y;
    const int pc = cell_off[kr.z] + kr.w;
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
    if (sr_lo) {   // float32 records carry the rounding residue (float-float local coordinates)
        Vec4<real> c;
        c.x = static_cast<real>(r.loc[0] - static_cast<double>(b.x));
        c.y = static_cast<real>(r.loc[1] - static_cast<double>(b.y));
        c.z = static_cast<real>(r.loc[2] - static_cast<double>(b.z));
        c.w = real(0);
        sr_lo[pc] = c;
    }
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

// ---- Alg. 2 step 1: spreading ------------------------------------------------------------------
// One CTA per tile of T^3 stencil-start bins.  Thread t owns the column (b, c) = (t / E, t % E) of
// the tile's extended block (E = T + P - 1 points per axis) and keeps its E values along the first
// axis in registers; every particle of the tile adds rho wy[b-oy] wz[c-oz] wx[.] to them.  The
// block is written to a per-tile scratch slab; k_halo sums overlapping slabs (no atomics anywhere).
constexpr int kSpreadChunk = 64;

template <int P>
constexpr int spread_threads() { return (((kTile + P - 1) * (kTile + P - 1) + 31) / 32) * 32; }

template <typename real, int P>
__global__ void __launch_bounds__(spread_threads<P>()) k_spread(const Vec4<real>* __restrict__ rec, const int2* __restrict__ idx,
                                                 const int* __restrict__ tile_off, const real* __restrict__ wcoef,
                                                 int degw, real* __restrict__ scratch) {
    constexpr int T = kTile, E = T + P - 1, CH = kSpreadChunk;
    const int tile = blockIdx.x;
    const int beg = tile_off[tile], end = tile_off[tile + 1];
    if (beg == end) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* sc = reinterpret_cast<real*>(smem_raw);                 // P * (degw + 1)
    real* sw = sc + P * (degw + 1);                                // CH * 3 * P
    real* srho = sw + CH * 3 * P;                                  // CH
    int* soff = reinterpret_cast<int*>(srho + CH);                 // CH
    for (int i = threadIdx.x; i < P * (degw + 1); i += blockDim.x) sc[i] = wcoef[i];

    const int col = threadIdx.x;
    const bool own = col < E * E;
    const int b = col / E, c = col % E;
    real acc[E];
#pragma unroll
    for (int a = 0; a < E; ++a) acc[a] = real(0);

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
            for (int a = 0; a < P; ++a) sw[(j * 3 + d) * P + a] = w[a];
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
                const real wyz = srho[j] * sw[(j * 3 + 1) * P + bb] * sw[(j * 3 + 2) * P + cc];
                const real* wx = sw + (j * 3) * P;
                switch (ox) {
#define PSWF_SPREAD_CASE(O)                                               \
    case O:                                                               \
        _Pragma("unroll") for (int p = 0; p < P; ++p) acc[O + p] = fma(wyz, wx[p], acc[O + p]); \
        break;
                    PSWF_SPREAD_CASE(0)
                    PSWF_SPREAD_CASE(1)
                    PSWF_SPREAD_CASE(2)
                    PSWF_SPREAD_CASE(3)
#undef PSWF_SPREAD_CASE
                    default: break;
                }
            }
        }
    }
    if (own) {
        real* out = scratch + static_cast<size_t>(tile) * E * E * E;
#pragma unroll
        for (int a = 0; a < E; ++a) out[a * E * E + col] = acc[a];
    }
}

// Sum of every tile slab covering grid point l (periodic): tile t, slab offset e with t T + e = l mod m.
template <typename real>
__global__ void k_halo(const real* __restrict__ scratch, const int* __restrict__ tile_off, Geom g,
                       real* __restrict__ grid) {
    const int m = g.m, T = g.T, nt = g.nt, E = g.T + g.P - 1;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= m * m * m) return;
    const int lz = id % m, ly = (id / m) % m, lx = id / (m * m);
    real s = real(0);
    for (int ex = 0; ex < E; ++ex) {
        int rx = (lx - ex) % m;
        if (rx < 0) rx += m;
        if (rx % T) continue;
        const int tx = rx / T;
        for (int ey = 0; ey < E; ++ey) {
            int ry = (ly - ey) % m;
            if (ry < 0) ry += m;
            if (ry % T) continue;
            const int ty = ry / T;
            for (int ez = 0; ez < E; ++ez) {
                int rz = (lz - ez) % m;
                if (rz < 0) rz += m;
                if (rz % T) continue;
                const int tz = rz / T;
                const int tile = (tx * nt + ty) * nt + tz;
                if (tile_off[tile] == tile_off[tile + 1]) continue;
                s += scratch[static_cast<size_t>(tile) * E * E * E + (ex * E + ey) * E + ez];
            }
        }
    }
    grid[id] = s;
}

// ---- Alg. 2 step 3: diagonal scaling on the R2C half spectrum ------------------------------------
template <typename real, typename cplx>
__global__ void k_scale(cplx* __restrict__ spec, int m, const real* __restrict__ iw, const real* __restrict__ mtab) {
    const int mh = m / 2 + 1;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= m * m * mh) return;
    const int iz = id % mh, iy = (id / mh) % m, ix = id / (mh * m);
    const int kx = ix < m / 2 ? ix : ix - m, ky = iy < m / 2 ? iy : iy - m, kz = iz;
    const int q = kx * kx + ky * ky + kz * kz;
    const int qmax = (m / 2) * (m / 2);
    real s = real(0);
    if (q > 0 && q < qmax) s = mtab[q] * iw[ix] * iw[iy] * iw[iz];   // open ball |k| < m/2
    cplx v = spec[id];
    v.x *= s;
    v.y *= s;
    spec[id] = v;
}

// ---- Alg. 2 step 5 with eq. force: interpolation of phi and grad phi ------------------------------
// One CTA per tile: the tile's extended block of the grid b (E^3 values) is staged in shared memory.
// Each warp first evaluates the 6 P window weights (value, derivative per axis) of NB particles,
// one particle per lane, then contracts each particle's P^3 stencil cooperatively: lanes take
// (b, c) pairs, reduce over a in registers, and the warp sums the four results by shuffles.
template <typename real> struct InterpCfg;
template <> struct InterpCfg<float> { static constexpr int NB = 32, NWARP = 4; };
template <> struct InterpCfg<double> { static constexpr int NB = 8, NWARP = 4; };

template <typename real, int P>
__global__ void __launch_bounds__(128) k_interp(const real* __restrict__ grid, const Vec4<real>* __restrict__ rec,
                                                const int2* __restrict__ idx, const int* __restrict__ tile_off,
                                                const real* __restrict__ wcoef, const real* __restrict__ dwcoef,
                                                Geom g, real inv_alpha, double* __restrict__ phi_out,
                                                double* __restrict__ f_out) {
    constexpr int T = kTile, E = T + P - 1;
    constexpr int NB = InterpCfg<real>::NB, NWARP = InterpCfg<real>::NWARP;
    const int tile = blockIdx.x;
    const int beg = tile_off[tile], end = tile_off[tile + 1];
    if (beg == end) return;
    const int m = g.m, nt = g.nt, degw = g.degw;
    const int tz = tile % nt, ty = (tile / nt) % nt, tx = tile / (nt * nt);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* G = reinterpret_cast<real*>(smem_raw);                 // E^3
    real* sc = G + E * E * E;                                     // P * (degw + 1)
    real* sd = sc + P * (degw + 1);                               // P * (degw + 1)
    real* sw = sd + P * (degw + 1);                               // NWARP * NB * 6 * P
    for (int i = threadIdx.x; i < P * (degw + 1); i += blockDim.x) {
        sc[i] = wcoef[i];
        sd[i] = dwcoef[i];
    }
    for (int e = threadIdx.x; e < E * E * E; e += blockDim.x) {
        const int ez = e % E, ey = (e / E) % E, ex = e / (E * E);
        const int gx = (tx * T + ex) % m, gy = (ty * T + ey) % m, gz = (tz * T + ez) % m;
        G[e] = grid[(static_cast<size_t>(gx) * m + gy) * m + gz];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    real* ww = sw + warp * NB * 6 * P;
    for (int b0 = beg + warp * NB; b0 < end; b0 += NWARP * NB) {
        const int cnt = min(NB, end - b0);
        __syncwarp();
        if (lane < cnt) {
            const Vec4<real> r = rec[b0 + lane];
            real w[P];
            const real zz[3] = {r.x, r.y, r.z};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                window_weights<real, P>(sc, degw, zz[d], w);
#pragma unroll
                for (int a = 0; a < P; ++a) ww[(lane * 6 + d) * P + a] = w[a];
                window_weights<real, P>(sd, degw, zz[d], w);
#pragma unroll
                for (int a = 0; a < P; ++a) ww[(lane * 6 + 3 + d) * P + a] = w[a] * inv_alpha;
            }
        }
        __syncwarp();
        for (int j = 0; j < cnt; ++j) {
            const int2 id = idx[b0 + j];
            const int ox = id.x & 0xff, oy = (id.x >> 8) & 0xff, oz = (id.x >> 16) & 0xff;
            const real* wp = ww + j * 6 * P;
            real wx[P], dwx[P];
#pragma unroll
            for (int a = 0; a < P; ++a) {
                wx[a] = wp[a];
                dwx[a] = wp[3 * P + a];
            }
            real ph = 0, gx = 0, gy = 0, gz = 0;
            for (int q = lane; q < P * P; q += 32) {
                const int bb = q / P, cc = q % P;
                const real* col = G + (ox * E + oy + bb) * E + oz + cc;
                real s1 = 0, s2 = 0;
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const real v = col[a * E * E];
                    s1 = fma(v, wx[a], s1);
                    s2 = fma(v, dwx[a], s2);
                }
                const real wy = wp[P + bb], wz = wp[2 * P + cc];
                const real dwy = wp[4 * P + bb], dwz = wp[5 * P + cc];
                const real yz = wy * wz;
                ph = fma(s1, yz, ph);
                gx = fma(s2, yz, gx);
                gy = fma(s1, dwy * wz, gy);
                gz = fma(s1, wy * dwz, gz);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ph += __shfl_xor_sync(0xffffffffu, ph, o);
                gx += __shfl_xor_sync(0xffffffffu, gx, o);
                gy += __shfl_xor_sync(0xffffffffu, gy, o);
                gz += __shfl_xor_sync(0xffffffffu, gz, o);
            }
            if (lane == 0) {
                const int i = id.y;
                const double q = static_cast<double>(rec[b0 + j].w);
                phi_out[i] = static_cast<double>(ph) - g.self * q;
                f_out[3 * static_cast<size_t>(i) + 0] = -q * static_cast<double>(gx);
                f_out[3 * static_cast<size_t>(i) + 1] = -q * static_cast<double>(gy);
                f_out[3 * static_cast<size_t>(i) + 2] = -q * static_cast<double>(gz);
            }
        }
    }
}

// ---- real-space sum of R over the cell list (Sec. 3.1.1) -----------------------------------------
// One thread per target in cell order; neighbour cells within `reach` whose box distance is below
// rc.  R(r) = 1/r - P1(u), -R'(r)/r = 1/r^3 + Q(u), u = 2 r^2/rc^2 - 1 (host-fitted polynomials).
// In float32 the pair displacement is formed in float-float: positions are (hi, lo) pairs relative
// to their cell, the neighbour-cell shift o is split the same way, and d = x_i - (x_j + o) is
// evaluated as (hi_i - (hi_j + o_hi)) + ((lo_i - o_lo) - lo_j): for close pairs across a cell face
// hi_j + o_hi cancels exactly, so d keeps full relative precision.
template <typename real>
__device__ __forceinline__ real rsqrt_r(real v);
template <> __device__ __forceinline__ float rsqrt_r<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_r<double>(double v) { return rsqrt(v); }

template <typename real>
__global__ void __launch_bounds__(128) k_short(const Vec4<real>* __restrict__ rec, const int2* __restrict__ idx,
                                               const Vec4<real>* __restrict__ lo, const int* __restrict__ cell_off,
                                               Geom g, const real* __restrict__ p1c, const real* __restrict__ qc,
                                               double* __restrict__ phi_out, double* __restrict__ f_out) {
    __shared__ real sp[64], sq[64];
    const int degr = g.degr;
    for (int k = threadIdx.x; k <= degr; k += blockDim.x) {
        sp[k] = p1c[k];
        sq[k] = qc[k];
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int nc = g.ncell, R = g.reach;
    const Vec4<real> me = rec[i];
    const Vec4<real> mlo = lo ? lo[i] : Vec4<real>{real(0), real(0), real(0), real(0)};
    const int2 id = idx[i];
    const int cz = id.x % nc, cy = (id.x / nc) % nc, cx = id.x / (nc * nc);
    const real rc2 = static_cast<real>(g.rc * g.rc);
    const real two_over_rc2 = static_cast<real>(2.0 / (g.rc * g.rc));
    const double cw2 = g.cellw * g.cellw, rcsq = g.rc * g.rc;
    real ph = 0, fx = 0, fy = 0, fz = 0;
    for (int dx = -R; dx <= R; ++dx) {
        const int bx = abs(dx) > 0 ? abs(dx) - 1 : 0;
        const double odx = dx * g.cellw;
        const real ohx = static_cast<real>(odx), olx = static_cast<real>(odx - static_cast<double>(ohx));
        for (int dy = -R; dy <= R; ++dy) {
            const int by = abs(dy) > 0 ? abs(dy) - 1 : 0;
            const double ody = dy * g.cellw;
            const real ohy = static_cast<real>(ody), oly = static_cast<real>(ody - static_cast<double>(ohy));
            for (int dz = -R; dz <= R; ++dz) {
                const int bz = abs(dz) > 0 ? abs(dz) - 1 : 0;
                if ((bx * bx + by * by + bz * bz) * cw2 >= rcsq) continue;
                const double odz = dz * g.cellw;
                const real ohz = static_cast<real>(odz), olz = static_cast<real>(odz - static_cast<double>(ohz));
                int nx = (cx + dx) % nc, ny = (cy + dy) % nc, nz = (cz + dz) % nc;
                nx += nx < 0 ? nc : 0;
                ny += ny < 0 ? nc : 0;
                nz += nz < 0 ? nc : 0;
                const int cell = (nx * nc + ny) * nc + nz;
                const int b = cell_off[cell], e = cell_off[cell + 1];
                const real lx = mlo.x - olx, ly = mlo.y - oly, lz = mlo.z - olz;
                for (int j = b; j < e; ++j) {
                    const Vec4<real> s = rec[j];
                    real ddx = me.x - (s.x + ohx), ddy = me.y - (s.y + ohy), ddz = me.z - (s.z + ohz);
                    if (lo) {
                        const Vec4<real> t = lo[j];
                        ddx += lx - t.x;
                        ddy += ly - t.y;
                        ddz += lz - t.z;
                    }
                    const real r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                    if (r2 < rc2 && r2 > real(0)) {
                        const real u = fma(r2, two_over_rc2, real(-1));
                        real p1 = sp[degr], q = sq[degr];
                        for (int k = degr - 1; k >= 0; --k) {
                            p1 = fma(p1, u, sp[k]);
                            q = fma(q, u, sq[k]);
                        }
                        const real ri = rsqrt_r<real>(r2);
                        ph = fma(s.w, ri - p1, ph);
                        const real cf = s.w * fma(ri * ri, ri, q);
                        fx = fma(cf, ddx, fx);
                        fy = fma(cf, ddy, fy);
                        fz = fma(cf, ddz, fz);
                    }
                }
            }
        }
    }
    const int o = id.y;
    const double qi = static_cast<double>(me.w);
    phi_out[o] += static_cast<double>(ph);
    f_out[3 * static_cast<size_t>(o) + 0] += qi * static_cast<double>(fx);
    f_out[3 * static_cast<size_t>(o) + 1] += qi * static_cast<double>(fy);
    f_out[3 * static_cast<size_t>(o) + 2] += qi * static_cast<double>(fz);
}

// ---- energy ------------------------------------------------------------------------------------
static __global__ void k_energy_partial(const double* __restrict__ phi, const double* __restrict__ rho, int n,
                                 double* __restrict__ part) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double q = rho[i];
        s += (isfinite(q) ? q : 0.0) * phi[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (warp == 0) {
        s = lane < (blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[blockIdx.x] = s;
    }
}

static __global__ void k_energy_final(const double* __restrict__ part, int np, double* __restrict__ energy) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
        energy[0] = 0.5 * t;
    }
}

}  // namespace pswf
