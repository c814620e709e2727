// Float-float kernels for tight tolerances: spreading, halo sum, interpolation and the real-space sum
// carried out in float-float arithmetic (ff.cuh) on the float32 pipes, about 48 significant bits; the
// grid, the FFTs and the scaling stay float64 (the float64 path's cuFFT plans and k_scale), and the
// outputs are float64.  Tiling, ownership and streaming are those of the kernels in device.cuh; only
// the arithmetic and the record layouts differ.  On this GPU float64 issues at ~1/64 of float32, so a
// float-float product (12-18 float32 operations) is several times cheaper than a float64 one.
//
// Inputs must lie in the float32 exponent range (|rho| and box sizes between ~1e-30 and ~1e30).
#pragma once

#include "device.cuh"
#include "ff.cuh"

namespace pswf {

__device__ __forceinline__ void split_ff(double v, float& h, float& l) {
    h = __double2float_rn(v);
    l = __double2float_rn(v - static_cast<double>(h));
}

// Sorted records.  Spreading side (tile order): {z0, z1, z2, rho} as separate high and low float4
// arrays, {packed offsets, original index}.  Real-space side (cell order): {local x, y, z, rho} high
// and low parts, {cell id, original index} and the cell's z index.
static __global__ void k_scatter_ff(const double* __restrict__ x, const double* __restrict__ rho, Geom g,
                                    const int* __restrict__ key_rank, const int* __restrict__ tile_off,
                                    const int* __restrict__ cell_off, float4* __restrict__ sp_h,
                                    float4* __restrict__ sp_l, int2* __restrict__ sp_idx, float4* __restrict__ sr_h,
                                    float4* __restrict__ sr_l, int2* __restrict__ sr_idx, int* __restrict__ sr_cz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const Located r = locate(x + 3 * static_cast<size_t>(i), g);
    double q = rho[i];
    if (!isfinite(q)) q = 0.0;
    const int4 kr = reinterpret_cast<const int4*>(key_rank)[i];
    const int ps = tile_off[kr.x] + kr.y;
    const int pc = cell_off[kr.z] + kr.w;
    float4 h, l;
    split_ff(r.z[0], h.x, l.x);
    split_ff(r.z[1], h.y, l.y);
    split_ff(r.z[2], h.z, l.z);
    split_ff(q, h.w, l.w);
    sp_h[ps] = h;
    sp_l[ps] = l;
    sp_idx[ps] = make_int2((r.lw[0] % g.T) | ((r.lw[1] % g.T) << 8) | ((r.lw[2] % g.T) << 16), i);
    split_ff(r.loc[0], h.x, l.x);
    split_ff(r.loc[1], h.y, l.y);
    split_ff(r.loc[2], h.z, l.z);
    sr_h[pc] = h;
    sr_l[pc] = l;
    sr_idx[pc] = make_int2(cell_of(r, g), i);
    sr_cz[pc] = r.cell[2];
}

// Window weight a at z (float-float).  The high-order terms k >= kf are tiny (the per-interval
// polynomials of the window decay fast) and are summed by a float32 Horner pass in z.h; the host picks
// kf so that pass stays well below the fit tolerance.  The terms k < kf run in float-float.
__device__ __forceinline__ ff window_weight_ff(const float* __restrict__ ch, const float* __restrict__ cl, int deg,
                                               int kf, int a, ff z) {
    const float* h = ch + a * (deg + 1);
    const float* l = cl + a * (deg + 1);
    float t = h[deg];
    for (int k = deg - 1; k >= kf; --k) t = fmaf(t, z.h, h[k]);
    ff w = ff_make(t);
    for (int k = kf - 1; k >= 0; --k) w = ff_horner_step(w, z, ff{h[k], l[k]});
    return ff_norm(w);
}

// ---- Alg. 2 step 1: spreading with float-float register columns, float2 {h, l} slabs ----------------
constexpr int kSpreadFFChunk = 32;

template <int P>
__global__ void __launch_bounds__(spread_threads<P, kTile64>()) k_spread_ff(const float4* __restrict__ rec_h,
                                                                   const float4* __restrict__ rec_l,
                                                                   const int2* __restrict__ idx,
                                                                   const int* __restrict__ tile_off,
                                                                   const float* __restrict__ wc, int degw, int kf,
                                                                   SpreadChain ch, float2* __restrict__ scratch) {
    constexpr int T = kTile64, E = T + P - 1, CH = kSpreadFFChunk;
    const int qx = blockIdx.x / ch.nyz, rem = blockIdx.x - qx * ch.nyz;   // chain: tiles (qx K + k, rem)
    const int nc = P * (degw + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ff* sw = reinterpret_cast<ff*>(smem_raw);                        // CH * 3 * P
    ff* srho = sw + CH * 3 * P;                                      // CH
    float* sch = reinterpret_cast<float*>(srho + CH);                // P * (degw + 1), then the low parts
    float* scl = sch + nc;
    int* soff = reinterpret_cast<int*>(scl + nc);                    // CH
    for (int i = threadIdx.x; i < 2 * nc; i += blockDim.x) sch[i] = wc[i];
    const int col = threadIdx.x;
    const bool own = col < E * E;
    const int b = col / E, c = col % E;
    ff acc[E];
#pragma unroll
    for (int a = 0; a < E; ++a) acc[a] = ff{0.f, 0.f};
    float2* heads = scratch;
    float2* tails = scratch + static_cast<size_t>(ch.ntiles) * T * E * E;
    for (int k = 0; k < ch.K; ++k) {
    const int tile = (qx * ch.K + k) * ch.nyz + rem;
    const int beg = tile_off[tile], end = tile_off[tile + 1];
    for (int base = beg; base < end; base += CH) {
        const int cnt = min(CH, end - base);
        __syncthreads();
        // one (particle, axis, weight) Horner evaluation per thread
        for (int t = threadIdx.x; t < cnt * 3 * P; t += blockDim.x) {
            const int j = t / (3 * P), d = (t / P) % 3, a = t % P;
            const float4 rh = rec_h[base + j], rl = rec_l[base + j];
            const ff z = d == 0 ? ff{rh.x, rl.x} : (d == 1 ? ff{rh.y, rl.y} : ff{rh.z, rl.z});
            sw[t] = window_weight_ff(sch, scl, degw, kf, a, z);
            if (d == 0 && a == 0) {
                srho[j] = ff{rh.w, rl.w};
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
                const ff wyz = ff_mul(ff_mul(srho[j], sw[(j * 3 + 1) * P + bb]), sw[(j * 3 + 2) * P + cc]);
                const ff* wx = sw + (j * 3) * P;
                switch (ox) {
#define PSWF_SPREAD_FF_CASE(O)                                                                \
    case O:                                                                                   \
        _Pragma("unroll") for (int p = 0; p < P; ++p) ff_acc(acc[O + p], wyz, wx[p]);        \
        break;
                    PSWF_SPREAD_FF_CASE(0)
                    PSWF_SPREAD_FF_CASE(1)
                    PSWF_SPREAD_FF_CASE(2)
                    PSWF_SPREAD_FF_CASE(3)
#undef PSWF_SPREAD_FF_CASE
                    default: break;
                }
            }
        }
    }
    if (own) {   // the tile's head (complete along x within the chain); carry the rest
        float2* out = heads + static_cast<size_t>(tile) * T * E * E;
#pragma unroll
        for (int a = 0; a < T; ++a) {
            const ff v = ff_norm(acc[a]);
            out[a * E * E + col] = make_float2(v.h, v.l);
        }
#pragma unroll
        for (int a = 0; a < E; ++a) acc[a] = a + T < E ? acc[a + T] : ff{0.f, 0.f};
    }
    }
    if (own) {   // the chain's tail
        float2* out = tails + static_cast<size_t>(blockIdx.x) * (E - T) * E * E;
#pragma unroll
        for (int a = 0; a < E - T; ++a) {
            const ff v = ff_norm(acc[a]);
            out[a * E * E + col] = make_float2(v.h, v.l);
        }
    }
}

// Halo sum of the float-float slabs (heads and x-chain tails, the enumeration of k_halo) into the
// float64 grid; the NZ overlapping z tiles are unrolled so their loads are in flight together.
template <int NZ>
__global__ void __launch_bounds__(256) k_halo_ff(const float2* __restrict__ scratch, const int* __restrict__ tile_off, Geom g,
                                                 double* __restrict__ grid) {
    (void)tile_off;
    const int my = g.m[1], mz = g.m[2], T = g.T, E = g.T + g.P - 1, ET = E - T;
    const int nty = g.nt[1], ntz = g.nt[2], K = g.K, nchx = g.nt[0] / g.K;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.m[0] * my * mz) return;
    const int lz = id % mz, ly = (id / mz) % my, lx = id / (mz * my);
    const int tlx = lx / T, tly = ly / T, tlz = lz / T;
    const int olx = lx - tlx * T, oly = ly - tly * T, olz = lz - tlz * T;
    const size_t plane = static_cast<size_t>(E) * E;
    const float2* heads = scratch;
    const float2* tails = scratch + static_cast<size_t>(g.nt[0]) * nty * ntz * T * plane;
    const int qc = tlx / K;
    int tzs[NZ];
#pragma unroll
    for (int c = 0; c < NZ; ++c) {   // tiny grids wrap repeatedly
        int t = tlz - c;
        while (t < 0) t += ntz;
        tzs[c] = t;
    }
    ff s{0.f, 0.f};
    int ty = tly;
    for (int ey = oly; ey < E; ey += T) {
        float2 v[NZ];
#pragma unroll
        for (int c = 0; c < NZ; ++c) {
            const int ez = olz + c * T;
            v[c] = make_float2(0.f, 0.f);
            if (ez < E)
                v[c] = heads[(static_cast<size_t>(tlx) * nty * ntz + ty * ntz + tzs[c]) * T * plane + olx * plane +
                             ey * E + ez];
        }
#pragma unroll
        for (int c = 0; c < NZ; ++c)
            if (olz + c * T < E) s = ff_add(s, ff{v[c].x, v[c].y});
        for (int j = 1;; ++j) {   // tails of the chains before this one that reach lx
            const int e = lx - (qc - j + 1) * K * T;
            if (e >= ET) break;
            int q = (qc - j) % nchx;
            q += q < 0 ? nchx : 0;
#pragma unroll
            for (int c = 0; c < NZ; ++c) {
                const int ez = olz + c * T;
                if (ez < E) {
                    const float2 w = tails[(static_cast<size_t>(q) * nty * ntz + ty * ntz + tzs[c]) * ET * plane +
                                           e * plane + ey * E + ez];
                    s = ff_add(s, ff{w.x, w.y});
                }
            }
        }
        ty = ty == 0 ? nty - 1 : ty - 1;
    }
    grid[id] = ff_to_double(s);
}

// float64 grid -> float-float pairs (after the inverse FFT, so the interpolation does no float64 work)
static __global__ void k_grid_to_ff(const double* __restrict__ grid, size_t count, float2* __restrict__ out) {
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float h, l;
    split_ff(grid[i], h, l);
    out[i] = make_float2(h, l);
}

// ---- Alg. 2 step 5 with eq. force: interpolation in float-float ------------------------------------
// Structure of k_interp (tile block in shared memory, a warp per batch of particles, lanes over the
// (b, c) pairs of the stencil); the inner sums over a are compensated dot products (ff_acc).
constexpr int kInterpFFNB = 4, kInterpFFWarps = 8;

// STAGED: the tile's extended block is staged in shared memory (E^3 float2); otherwise the grid is read
// through L1/L2 (it is L2-resident at these sizes) with per-particle wrapped index tables, so the block
// needs little shared memory and occupancy is set by registers.
template <int P, bool STAGED>
__global__ void __launch_bounds__(32 * kInterpFFWarps) k_interp_ff(const float2* __restrict__ grid,
                                                                   const float4* __restrict__ rec_h,
                                                                   const float4* __restrict__ rec_l,
                                                                   const int2* __restrict__ idx,
                                                                   const int* __restrict__ tile_off,
                                                                   const float* __restrict__ wc,
                                                                   const float* __restrict__ dwc, int kf, Geom g,
                                                                   float4 inv_alpha_h, float4 inv_alpha_l,
                                                                   double* __restrict__ phi_out,
                                                                   double* __restrict__ f_out) {
    constexpr int T = kTile64, E = T + P - 1, NB = kInterpFFNB, NWARP = kInterpFFWarps;
    constexpr int NQ = (P * P + 31) / 32;
    const int tile = blockIdx.x;
    const int beg = tile_off[tile], end = tile_off[tile + 1];
    if (beg == end) return;
    const int mx = g.m[0], my = g.m[1], mz = g.m[2], degw = g.degw;
    const int nc = P * (degw + 1);
    const int tz = tile % g.nt[2], ty = (tile / g.nt[2]) % g.nt[1], tx = tile / (g.nt[2] * g.nt[1]);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ff* G = reinterpret_cast<ff*>(smem_raw);                          // E^3 (STAGED only)
    ff* sw = G + (STAGED ? E * E * E : 0);                            // NWARP * NB * 6 * P
    float* sch = reinterpret_cast<float*>(sw + NWARP * NB * 6 * P);   // window hi, lo, derivative hi, lo
    float* scl = sch + nc;
    float* sdh = scl + nc;
    float* sdl = sdh + nc;
    for (int i = threadIdx.x; i < 2 * nc; i += blockDim.x) {
        sch[i] = wc[i];
        sdh[i] = dwc[i];
    }
    __shared__ int sxo[NWARP][P], syo[NWARP][P], szo[NWARP][P];   // unstaged: wrapped grid offsets
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (STAGED) {
        // z-rows of the block in 16-byte vectors (two float2 values) where they do not cross the periodic
        // end (rows start on 32-byte boundaries: z0 = 4 tz, m_z a multiple of 4); element-wise otherwise
        constexpr int NV = (E + 1) / 2, RPW = 32 / NV;
        const int z0 = tz * T;
        auto wrap = [](int v, int m) {
            while (v >= m) v -= m;
            return v;
        };
        if (z0 + 2 * NV <= mz) {
            const int rl = lane / NV, k = lane - rl * NV;
            for (int r0 = warp * RPW; r0 < E * E; r0 += NWARP * RPW) {
                const int row = r0 + rl;   // ex E + ey
                if (rl < RPW && row < E * E) {
                    const int ex = row / E, ey = row - ex * E;
                    const int gx = wrap(tx * T + ex, mx), gy = wrap(ty * T + ey, my);
                    const float4 v =
                        reinterpret_cast<const float4*>(grid + (static_cast<size_t>(gx) * my + gy) * mz + z0)[k];
                    ff* dst = G + row * E + 2 * k;
                    dst[0] = ff{v.x, v.y};
                    if (2 * k + 1 < E) dst[1] = ff{v.z, v.w};
                }
            }
        } else {
            for (int e = threadIdx.x; e < E * E * E; e += blockDim.x) {
                const int ez = e % E, ey = (e / E) % E, ex = e / (E * E);
                const int gx = wrap(tx * T + ex, mx), gy = wrap(ty * T + ey, my), gz = wrap(z0 + ez, mz);
                const float2 v = grid[(static_cast<size_t>(gx) * my + gy) * mz + gz];
                G[e] = ff{v.x, v.y};
            }
        }
    }
    __syncthreads();

    ff* ww = sw + warp * NB * 6 * P;
    for (int b0 = beg + warp * NB; b0 < end; b0 += NWARP * NB) {
        const int cnt = min(NB, end - b0);
        __syncwarp();
        // one (particle, kind, weight) Horner evaluation per lane; kinds 0-2 values, 3-5 derivatives
        for (int task = lane; task < cnt * 6 * P; task += 32) {
            const int j = task / (6 * P), kind = (task / P) % 6, a = task % P, d = kind % 3;
            const float4 rh = rec_h[b0 + j], rl = rec_l[b0 + j];
            const ff z = d == 0 ? ff{rh.x, rl.x} : (d == 1 ? ff{rh.y, rl.y} : ff{rh.z, rl.z});
            ww[task] = kind < 3 ? window_weight_ff(sch, scl, degw, kf, a, z)
                                : ff_mul(window_weight_ff(sdh, sdl, degw, kf, a, z),
                                         d == 0 ? ff{inv_alpha_h.x, inv_alpha_l.x}
                                                : (d == 1 ? ff{inv_alpha_h.y, inv_alpha_l.y} : ff{inv_alpha_h.z, inv_alpha_l.z}));
        }
        __syncwarp();
        ff mph{0.f, 0.f}, mgx{0.f, 0.f}, mgy{0.f, 0.f}, mgz{0.f, 0.f};   // lane j keeps particle j
        for (int j = 0; j < cnt; ++j) {
            const int2 id = idx[b0 + j];
            const int ox = id.x & 0xff, oy = (id.x >> 8) & 0xff, oz = (id.x >> 16) & 0xff;
            const ff* wp = ww + j * 6 * P;
            int xo[P];
            if constexpr (!STAGED) {   // wrapped row offsets of the particle's stencil
                __syncwarp();
                if (lane < P) {
                    sxo[warp][lane] = ((tx * T + ox + lane) % mx) * my * mz;
                    syo[warp][lane] = ((ty * T + oy + lane) % my) * mz;
                    szo[warp][lane] = (tz * T + oz + lane) % mz;
                }
                __syncwarp();
#pragma unroll
                for (int a = 0; a < P; ++a) xo[a] = sxo[warp][a];
            }
            ff ph{0.f, 0.f}, gx{0.f, 0.f}, gy{0.f, 0.f}, gz{0.f, 0.f};
#pragma unroll 1
            for (int qi = 0; qi < NQ; ++qi) {   // not unrolled: the a-loop body is already P x 48 instructions
                const int q = lane + 32 * qi;
                if (q < P * P) {
                    const int bb = q / P, cc = q - (q / P) * P;
                    auto at = [&](int a) -> ff {
                        if constexpr (STAGED) {
                            return G[((ox + a) * E + oy + bb) * E + oz + cc];
                        } else {
                            const float2 v = __ldg(grid + xo[a] + syo[warp][bb] + szo[warp][cc]);
                            return ff{v.x, v.y};
                        }
                    };
                    // four independent compensated chains (even / odd a) for instruction-level parallelism
                    ff s1a{0.f, 0.f}, s1b{0.f, 0.f}, s2a{0.f, 0.f}, s2b{0.f, 0.f};
#pragma unroll
                    for (int a = 0; a < P; a += 2) {
                        const ff v = at(a);
                        ff_acc(s1a, v, wp[a]);
                        ff_acc(s2a, v, wp[3 * P + a]);
                        if (a + 1 < P) {
                            const ff v2 = at(a + 1);
                            ff_acc(s1b, v2, wp[a + 1]);
                            ff_acc(s2b, v2, wp[3 * P + a + 1]);
                        }
                    }
                    const ff s1 = ff_add(ff_norm(s1a), ff_norm(s1b));
                    const ff s2 = ff_add(ff_norm(s2a), ff_norm(s2b));
                    const ff wy = wp[P + bb], wz = wp[2 * P + cc];
                    const ff dwy = wp[4 * P + bb], dwz = wp[5 * P + cc];
                    const ff yz = ff_mul(wy, wz);
                    ff_acc(ph, s1, yz);
                    ff_acc(gx, s2, yz);
                    ff_acc(gy, s1, ff_mul(dwy, wz));
                    ff_acc(gz, s1, ff_mul(wy, dwz));
                }
            }
            ph = ff_norm(ph);
            gx = ff_norm(gx);
            gy = ff_norm(gy);
            gz = ff_norm(gz);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ph = ff_add(ph, ff_shfl_xor(ph, o));
                gx = ff_add(gx, ff_shfl_xor(gx, o));
                gy = ff_add(gy, ff_shfl_xor(gy, o));
                gz = ff_add(gz, ff_shfl_xor(gz, o));
            }
            if (lane == j) {
                mph = ph;
                mgx = gx;
                mgy = gy;
                mgz = gz;
            }
        }
        if (lane < cnt) {   // float64 outputs, lane-parallel
            const int i = idx[b0 + lane].y;
            const double q = static_cast<double>(rec_h[b0 + lane].w) + static_cast<double>(rec_l[b0 + lane].w);
            phi_out[i] = ff_to_double(mph) - g.self * q;
            f_out[3 * static_cast<size_t>(i) + 0] = -q * ff_to_double(mgx);
            f_out[3 * static_cast<size_t>(i) + 1] = -q * ff_to_double(mgy);
            f_out[3 * static_cast<size_t>(i) + 2] = -q * ff_to_double(mgz);
        }
    }
}

// ---- real-space sum of R in float-float ---------------------------------------------------------
// Cell traversal of k_short (a warp per target cell, flattened neighbour ranges) in the two-phase form
// of k_short_q, since one float-float pair costs ~40x a float32 cutoff test: the float32 scan fills
// per-target pair queues, and full warps of queued pairs are evaluated in float-float: the
// displacement d = (hi_i - (hi_j + s_hi)) + (lo_i - (lo_j + s_lo)) with the leading difference and the
// cell shift split exactly (TwoSum), R and -R'/r from the radial polynomials by Horner (float32 for
// the tiny leading terms k >= kr, float-float below), 1/r from a float32 estimate with a float-float
// correction, and compensated accumulation.  The pair evaluation exists once in the code.
constexpr int kShortFFMaxT = 4;   // targets per pass (float-float sums in registers: 32 of them)

// Radial polynomials padded with zeros to degree D; terms k >= kr (tiny, chosen on the host) are summed
// by float32 Horner steps in u.h, the terms below kr in float-float.
template <int D>
struct ShortParamsFF {
    float p1h[D + 1], p1l[D + 1], qh[D + 1], ql[D + 1];
    float rc2h, rc2l, two_over_rc2_h, two_over_rc2_l;
    float rc2f;
    int kr;
};

// acc += c for an unnormalised accumulator (error terms collected in acc.l)
__device__ __forceinline__ void ff_acc_sum(ff& acc, ff c) {
    const ff s = two_sum(acc.h, c.h);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, c.l));
}

template <int D>
__global__ void __launch_bounds__(32 * kShortWarps, 6) k_short_ff(const float4* __restrict__ rec_h,
                                                                  const float4* __restrict__ rec_l,
                                                                  const int2* __restrict__ idx,
                                                                  const int* __restrict__ cz_of,
                                                                  const int* __restrict__ cell_off,
                                                                  const int4* __restrict__ cols, int ncols, int rcap,
                                                                  Geom g, const __grid_constant__ ShortParamsFF<D> kp,
                                                                  double* __restrict__ phi_out,
                                                                  double* __restrict__ f_out) {
    constexpr int NSH = 2 * kShortMaxR + 1, MT = kShortFFMaxT;
    static_assert(NSH <= 16, "queue entries pack 4-bit shift indices");
    __shared__ float sh_hi[3][NSH], sh_lo[3][NSH];   // cell shifts (k - R) w_d, hi and lo parts
    __shared__ int4 scol[(2 * kShortMaxR + 1) * (2 * kShortMaxR + 1)];
    __shared__ float4 sth[kShortWarps][MT], stl[kShortWarps][MT];
    __shared__ int2 sq[kShortWarps][MT][kShortQCap];   // {source, ix | iy << 4 | iz << 8}
    __shared__ int sqlen[kShortWarps][MT];
    const int R = g.reach, Rz = g.reachz;
    for (int k = threadIdx.x; k < 3 * NSH; k += blockDim.x) {
        const int d = k / NSH, i = k % NSH, rd = d == 2 ? Rz : R;
        split_ff((i - rd) * g.cellw[d], sh_hi[d][i], sh_lo[d][i]);
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

    const ff rc2{kp.rc2h, kp.rc2l}, two_over_rc2{kp.two_over_rc2_h, kp.two_over_rc2_l};
    for (int t0 = tb; t0 < te; t0 += MT) {
        const int nt = min(MT, te - t0);
        __syncwarp();
        if (lane < nt) {
            sth[warp][lane] = rec_h[t0 + lane];
            stl[warp][lane] = rec_l[t0 + lane];
        }
        if (lane < MT) qlen[lane] = 0;
        __syncwarp();
        ff acc[MT][4];
#pragma unroll
        for (int t = 0; t < MT; ++t)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[t][v] = ff{0.f, 0.f};

        // one queued pair for target t (warp-uniform) -> the lane's sums of that target
        auto pair = [&](int2 e, int t, bool active) {
            const int ix = e.y & 15, iy = (e.y >> 4) & 15, iz = (e.y >> 8) & 15;
            const int j = active ? e.x : t0;
            const float4 sh = rec_h[j], sl = rec_l[j];
            const float4 th = sth[warp][t], tl = stl[warp][t];
            const ff ex = two_sum(sh.x, sh_hi[0][ix]), ey = two_sum(sh.y, sh_hi[1][iy]), ez = two_sum(sh.z, sh_hi[2][iz]);
            const float lx = __fadd_rn(__fadd_rn(sl.x, sh_lo[0][ix]), ex.l);
            const float ly = __fadd_rn(__fadd_rn(sl.y, sh_lo[1][iy]), ey.l);
            const float lz = __fadd_rn(__fadd_rn(sl.z, sh_lo[2][iz]), ez.l);
            ff dx = two_sum(th.x, -ex.h), dy = two_sum(th.y, -ey.h), dz = two_sum(th.z, -ez.h);
            dx = two_sum(dx.h, __fadd_rn(dx.l, __fadd_rn(tl.x, -lx)));
            dy = two_sum(dy.h, __fadd_rn(dy.l, __fadd_rn(tl.y, -ly)));
            dz = two_sum(dz.h, __fadd_rn(dz.l, __fadd_rn(tl.z, -lz)));
            const ff r2 = ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
            const bool in = active && (r2.h < rc2.h || (r2.h == rc2.h && r2.l < rc2.l)) && r2.h > 0.f;
            const ff u = ff_add(ff_mul(r2, two_over_rc2), ff_make(-1.f));
            float p1f = kp.p1h[D], qqf = kp.qh[D];
            ff p1 = ff_make(p1f), qq = ff_make(qqf);
#pragma unroll
            for (int kk = D - 1; kk >= 0; --kk) {
                if (kk >= kp.kr) {   // warp-uniform
                    p1f = fmaf(p1f, u.h, kp.p1h[kk]);
                    qqf = fmaf(qqf, u.h, kp.qh[kk]);
                    p1 = ff_make(p1f);
                    qq = ff_make(qqf);
                } else {
                    p1 = ff_horner_step(p1, u, ff{kp.p1h[kk], kp.p1l[kk]});
                    qq = ff_horner_step(qq, u, ff{kp.qh[kk], kp.ql[kk]});
                }
            }
            p1 = ff_norm(p1);
            qq = ff_norm(qq);
            const ff ri = ff_rsqrt(in ? r2 : ff_make(1.f));
            const ff qj = in ? ff{sh.w, sl.w} : ff{0.f, 0.f};
            const ff c0 = ff_mul(qj, ff_sub(ri, p1));
            const ff cf = ff_mul(qj, ff_add(ff_mul(ff_sqr(ri), ri), qq));
            const ff c1 = ff_mul(cf, dx), c2 = ff_mul(cf, dy), c3 = ff_mul(cf, dz);
#pragma unroll
            for (int tt = 0; tt < MT; ++tt)
                if (tt == t) {   // warp-uniform
                    ff_acc_sum(acc[tt][0], c0);
                    ff_acc_sum(acc[tt][1], c1);
                    ff_acc_sum(acc[tt][2], c2);
                    ff_acc_sum(acc[tt][3], c3);
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
                    const float4 sh = rec_h[j];
                    const int4 col = scol[rg.w];
                    const int ix = col.x + R, iy = col.y + R, iz = rg.z + (cz_of[j] - rg.y) + Rz;
                    const float px = sh.x + sh_hi[0][ix], py = sh.y + sh_hi[1][iy], pz = sh.z + sh_hi[2][iz];
#pragma unroll
                    for (int t = 0; t < MT; ++t) {
                        if (t >= nt) break;   // warp-uniform
                        const float4 a = sth[warp][t];
                        const float dxf = a.x - px, dyf = a.y - py, dzf = a.z - pz;
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

        // reduce each target's sums over the lanes; lane t writes target t
#pragma unroll
        for (int t = 0; t < MT; ++t)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                ff x = ff_norm(acc[t][v]);
                for (int o = 16; o > 0; o >>= 1) x = ff_add(x, ff_shfl_xor(x, o));
                acc[t][v] = x;
            }
        ff mine[4] = {ff{0.f, 0.f}, ff{0.f, 0.f}, ff{0.f, 0.f}, ff{0.f, 0.f}};
#pragma unroll
        for (int t = 0; t < MT; ++t)
            if (lane == t) {
                mine[0] = acc[t][0];
                mine[1] = acc[t][1];
                mine[2] = acc[t][2];
                mine[3] = acc[t][3];
            }
        if (lane < nt) {   // float64 conversions once per pass, lane-parallel
            const int oi = idx[t0 + lane].y;
            const double qi = static_cast<double>(sth[warp][lane].w) + static_cast<double>(stl[warp][lane].w);
            phi_out[oi] = ff_to_double(mine[0]);
            f_out[3 * static_cast<size_t>(oi) + 0] = qi * ff_to_double(mine[1]);
            f_out[3 * static_cast<size_t>(oi) + 1] = qi * ff_to_double(mine[2]);
            f_out[3 * static_cast<size_t>(oi) + 2] = qi * ff_to_double(mine[3]);
        }
        __syncwarp();
    }
}

}  // namespace pswf
