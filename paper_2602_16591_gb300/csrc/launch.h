// Host-side launchers for the P-templated kernels (one translation unit per precision).
#pragma once

#include <cuda_runtime.h>

#include "device.cuh"

namespace pswf {

constexpr int kPMin = 3, kPMax = 24;

template <typename real>
struct Launch {
    static size_t spread_smem(int P, int degw);
    static size_t interp_smem(int P, int degw);
    // ch: x-chains of ch.K tiles (grid of ntiles / ch.K blocks), slab layout of k_spread
    static cudaError_t spread(int P, int ntiles, const Vec4<real>* rec, const int2* idx, const int* tile_off,
                              const real* wcoef, int degw, SpreadChain ch, real* scratch, cudaStream_t s);
    static cudaError_t interp(int P, int ntiles, const real* grid, const Vec4<real>* rec, const int2* idx,
                              const int* tile_off, const real* wcoef, const real* dwcoef, const Geom& g,
                              Vec4<real> inv_alpha, double* phi, double* f, cudaStream_t s);
};

// Float-float path (dispatch_ff.cu): float-float records, spreading, interpolation and real-space sum;
// float64 grid, FFT and scaling.  Window tables hold P * (deg_w + 1) high parts followed by as many low
// parts; terms k >= kf of the window polynomials are summed in float32.
struct LaunchFF {
    static cudaError_t scatter(const double* x, const double* rho, const Geom& g, const int* key_rank,
                               const int* tile_off, const int* cell_off, float4* sp_h, float4* sp_l, int2* sp_idx,
                               float4* sr_h, float4* sr_l, int2* sr_idx, int* sr_cz, cudaStream_t s);
    static cudaError_t spread(int ntiles, const Geom& g, const float4* rec_h, const float4* rec_l, const int2* idx,
                              const int* tile_off, const float* wc, int kf, float2* scratch, cudaStream_t s);
    static cudaError_t halo(const float2* scratch, const int* tile_off, const Geom& g, double* grid, cudaStream_t s);
    static cudaError_t to_ff(const double* grid, size_t count, float2* out, cudaStream_t s);
    static cudaError_t interp(int ntiles, const Geom& g, const float2* grid, const float4* rec_h, const float4* rec_l,
                              const int2* idx, const int* tile_off, const float* wc, const float* dwc, int kf,
                              const double* inv_alpha, double* phi, double* f, cudaStream_t s);
    // radial polynomials p1c / qc of degree g.degr (float64 coefficients, split on the host); terms
    // k >= kr are summed in float32
    static cudaError_t short_range(const Geom& g, const float4* rec_h, const float4* rec_l, const int2* idx,
                                   const int* cz, const int* cell_off, const int4* cols, int ncols, int rcap,
                                   const double* p1c, const double* qc, int kr, double* phi, double* f, cudaStream_t s);
};

}  // namespace pswf
