// Launchers of the float-float kernels (ff_kernels.cuh): P- and degree-templated instantiations and
// their runtime dispatch.
#include "ff_kernels.cuh"
#include "launch.h"

namespace pswf {

namespace {

void split(double v, float& h, float& l) {
    h = static_cast<float>(v);
    l = static_cast<float>(v - static_cast<double>(h));
}

size_t spread_smem_ff(int P, int degw) {
    return sizeof(ff) * (kSpreadFFChunk * 3 * P + kSpreadFFChunk) + sizeof(float) * 2 * P * (degw + 1) +
           sizeof(int) * kSpreadFFChunk;
}

size_t interp_smem_ff(int P, int degw, bool staged) {
    const int E = kTile64 + P - 1;
    return sizeof(ff) * ((staged ? static_cast<size_t>(E) * E * E : 0) + kInterpFFWarps * kInterpFFNB * 6 * P) +
           sizeof(float) * 4 * P * (degw + 1);
}

template <int P>
cudaError_t spread_p(int ntiles, const Geom& g, const float4* rh, const float4* rl, const int2* idx,
                     const int* tile_off, const float* wc, int kf, float2* scratch, cudaStream_t s) {
    const size_t smem = spread_smem_ff(P, g.degw);
    auto kern = k_spread_ff<P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const SpreadChain ch{g.K, g.nt[1] * g.nt[2], ntiles};
    kern<<<ntiles / g.K, spread_threads<P, kTile64>(), smem, s>>>(rh, rl, idx, tile_off, wc, g.degw, kf, ch, scratch);
    return cudaGetLastError();
}

template <int P>
cudaError_t interp_p(int ntiles, const Geom& g, const float2* grid, const float4* rh, const float4* rl,
                     const int2* idx, const int* tile_off, const float* wc, const float* dwc, int kf, float4 iah,
                     float4 ial, double* phi, double* f, cudaStream_t s) {
    // stage the tile's block while two blocks still fit an SM (measured: staged wins at P = 16, direct
    // L1/L2 reads win at P = 19, where a staged block allows one block per SM)
    const bool staged = interp_smem_ff(P, g.degw, true) <= 113 * 1024;
    const size_t smem = interp_smem_ff(P, g.degw, staged);
    auto kern = staged ? k_interp_ff<P, true> : k_interp_ff<P, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<ntiles, 32 * kInterpFFWarps, smem, s>>>(grid, rh, rl, idx, tile_off, wc, dwc, kf, g, iah, ial, phi, f);
    return cudaGetLastError();
}

template <int D>
cudaError_t short_d(const Geom& g, const float4* rh, const float4* rl, const int2* idx, const int* cz,
                    const int* cell_off, const int4* cols, int ncols, int rcap, const double* p1c, const double* qc,
                    int kr, double* phi, double* f, cudaStream_t s) {
    ShortParamsFF<D> kp{};
    for (int k = 0; k <= D; ++k) {
        split(k <= g.degr ? p1c[k] : 0.0, kp.p1h[k], kp.p1l[k]);
        split(k <= g.degr ? qc[k] : 0.0, kp.qh[k], kp.ql[k]);
    }
    split(g.rc * g.rc, kp.rc2h, kp.rc2l);
    split(2.0 / (g.rc * g.rc), kp.two_over_rc2_h, kp.two_over_rc2_l);
    kp.rc2f = static_cast<float>(g.rc * g.rc * (1.0 + 1e-4));
    kp.kr = kr;
    const int ncells = g.ncell[0] * g.ncell[1] * g.ncell[2];
    const size_t smem = short_dyn_smem(rcap);
    k_short_ff<D><<<(ncells + kShortWarps - 1) / kShortWarps, 32 * kShortWarps, smem, s>>>(
        rh, rl, idx, cz, cell_off, cols, ncols, rcap, g, kp, phi, f);
    return cudaGetLastError();
}

}  // namespace

#define PSWF_FF_P_CASES(X) \
    X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24)

cudaError_t LaunchFF::scatter(const double* x, const double* rho, const Geom& g, const int* key_rank,
                              const int* tile_off, const int* cell_off, float4* sp_h, float4* sp_l, int2* sp_idx,
                              float4* sr_h, float4* sr_l, int2* sr_idx, int* sr_cz, cudaStream_t s) {
    const int tb = 256, nb = (g.n + tb - 1) / tb;
    k_scatter_ff<<<nb, tb, 0, s>>>(x, rho, g, key_rank, tile_off, cell_off, sp_h, sp_l, sp_idx, sr_h, sr_l, sr_idx,
                                   sr_cz);
    return cudaGetLastError();
}

cudaError_t LaunchFF::spread(int ntiles, const Geom& g, const float4* rec_h, const float4* rec_l, const int2* idx,
                             const int* tile_off, const float* wc, int kf, float2* scratch, cudaStream_t s) {
    switch (g.P) {
#define X(p) case p: return spread_p<p>(ntiles, g, rec_h, rec_l, idx, tile_off, wc, kf, scratch, s);
        PSWF_FF_P_CASES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t LaunchFF::halo(const float2* scratch, const int* tile_off, const Geom& g, double* grid, cudaStream_t s) {
    const int mm = g.m[0] * g.m[1] * g.m[2];
    const int nz = (g.T + g.P - 1 + g.T - 1) / g.T, hb = (mm + 255) / 256;   // overlapping slabs per axis
    if (nz <= 4) k_halo_ff<4><<<hb, 256, 0, s>>>(scratch, tile_off, g, grid);
    else if (nz <= 6) k_halo_ff<6><<<hb, 256, 0, s>>>(scratch, tile_off, g, grid);
    else if (nz <= 8) k_halo_ff<8><<<hb, 256, 0, s>>>(scratch, tile_off, g, grid);
    else if (nz <= 16) k_halo_ff<16><<<hb, 256, 0, s>>>(scratch, tile_off, g, grid);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t LaunchFF::to_ff(const double* grid, size_t count, float2* out, cudaStream_t s) {
    k_grid_to_ff<<<static_cast<unsigned>((count + 255) / 256), 256, 0, s>>>(grid, count, out);
    return cudaGetLastError();
}

cudaError_t LaunchFF::interp(int ntiles, const Geom& g, const float2* grid, const float4* rec_h, const float4* rec_l,
                             const int2* idx, const int* tile_off, const float* wc, const float* dwc, int kf,
                             const double* inv_alpha, double* phi, double* f, cudaStream_t s) {
    float4 iah{}, ial{};
    split(inv_alpha[0], iah.x, ial.x);
    split(inv_alpha[1], iah.y, ial.y);
    split(inv_alpha[2], iah.z, ial.z);
    switch (g.P) {
#define X(p) case p: return interp_p<p>(ntiles, g, grid, rec_h, rec_l, idx, tile_off, wc, dwc, kf, iah, ial, phi, f, s);
        PSWF_FF_P_CASES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t LaunchFF::short_range(const Geom& g, const float4* rec_h, const float4* rec_l, const int2* idx,
                                  const int* cz, const int* cell_off, const int4* cols, int ncols, int rcap,
                                  const double* p1c, const double* qc, int kr, double* phi, double* f, cudaStream_t s) {
    const int d = g.degr;
    if (d <= 8) return short_d<8>(g, rec_h, rec_l, idx, cz, cell_off, cols, ncols, rcap, p1c, qc, kr, phi, f, s);
    if (d <= 12) return short_d<12>(g, rec_h, rec_l, idx, cz, cell_off, cols, ncols, rcap, p1c, qc, kr, phi, f, s);
    if (d <= 16) return short_d<16>(g, rec_h, rec_l, idx, cz, cell_off, cols, ncols, rcap, p1c, qc, kr, phi, f, s);
    if (d <= 20) return short_d<20>(g, rec_h, rec_l, idx, cz, cell_off, cols, ncols, rcap, p1c, qc, kr, phi, f, s);
    if (d <= 24) return short_d<24>(g, rec_h, rec_l, idx, cz, cell_off, cols, ncols, rcap, p1c, qc, kr, phi, f, s);
    if (d <= 32) return short_d<32>(g, rec_h, rec_l, idx, cz, cell_off, cols, ncols, rcap, p1c, qc, kr, phi, f, s);
    if (d <= 44) return short_d<44>(g, rec_h, rec_l, idx, cz, cell_off, cols, ncols, rcap, p1c, qc, kr, phi, f, s);
    return short_d<60>(g, rec_h, rec_l, idx, cz, cell_off, cols, ncols, rcap, p1c, qc, kr, phi, f, s);
}

}  // namespace pswf
