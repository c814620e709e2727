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
    static cudaError_t spread(int P, int ntiles, const Vec4<real>* rec, const int2* idx, const int* tile_off,
                              const real* wcoef, int degw, real* scratch, cudaStream_t s);
    static cudaError_t interp(int P, int ntiles, const real* grid, const Vec4<real>* rec, const int2* idx,
                              const int* tile_off, const real* wcoef, const real* dwcoef, const Geom& g,
                              real inv_alpha, double* phi, double* f, cudaStream_t s);
};

}  // namespace pswf
