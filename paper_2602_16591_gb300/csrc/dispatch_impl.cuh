// Instantiates the P-templated spreading and interpolation kernels for one precision `real_t`
// (included by dispatch_f32.cu / dispatch_f64.cu) and dispatches a runtime P to them.
#include "launch.h"

namespace pswf {

namespace {

template <int P>
cudaError_t spread_p(int ntiles, const Vec4<real_t>* rec, const int2* idx, const int* tile_off, const real_t* wcoef,
                     int degw, SpreadChain ch, real_t* scratch, cudaStream_t s) {
    const int threads = spread_threads<P, spread_tile<real_t>()>();
    const size_t smem = Launch<real_t>::spread_smem(P, degw);
    auto kern = k_spread<real_t, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<ntiles / ch.K, threads, smem, s>>>(rec, idx, tile_off, wcoef, degw, ch, scratch);
    return cudaGetLastError();
}

template <int P>
cudaError_t interp_p(int ntiles, const real_t* grid, const Vec4<real_t>* rec, const int2* idx, const int* tile_off,
                     const real_t* wcoef, const real_t* dwcoef, const Geom& g, Vec4<real_t> inv_alpha, double* phi, double* f,
                     cudaStream_t s) {
    const size_t smem = Launch<real_t>::interp_smem(P, g.degw);
    auto kern = k_interp<real_t, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<ntiles, 32 * InterpCfg<real_t>::NWARP, smem, s>>>(grid, rec, idx, tile_off, wcoef, dwcoef, g, inv_alpha,
                                                          phi, f);
    return cudaGetLastError();
}

}  // namespace

template <>
size_t Launch<real_t>::spread_smem(int P, int degw) {
    constexpr int VW = 16 / static_cast<int>(sizeof(real_t));
    const int PP = (P + VW - 1) / VW * VW;   // padded weight rows (k_spread)
    return sizeof(real_t) * (kSpreadChunk * 3 * PP + P * (degw + 1) + kSpreadChunk) + sizeof(int) * kSpreadChunk;
}

template <>
size_t Launch<real_t>::interp_smem(int P, int degw) {
    const int E = spread_tile<real_t>() + P - 1;
    constexpr int VW = 16 / static_cast<int>(sizeof(real_t));
    const int PP = (P + VW - 1) / VW * VW;   // padded weight rows (k_interp)
    const int SP = E * E + (((P - E * E) % 32) + 32) % 32;   // padded y-plane (k_interp)
    const size_t block = (static_cast<size_t>(E) * SP + VW - 1) / VW * VW;   // staged block, then coefficient rows
    return sizeof(real_t) * (block + 2 * static_cast<size_t>(PP) * (degw + 1) +
                             InterpCfg<real_t>::NWARP * InterpCfg<real_t>::NB * 6 * PP);
}

#define PSWF_P_CASES(X) \
    X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24)

template <>
cudaError_t Launch<real_t>::spread(int P, int ntiles, const Vec4<real_t>* rec, const int2* idx, const int* tile_off,
                                 const real_t* wcoef, int degw, SpreadChain ch, real_t* scratch, cudaStream_t s) {
    switch (P) {
#define X(p) case p: return spread_p<p>(ntiles, rec, idx, tile_off, wcoef, degw, ch, scratch, s);
        PSWF_P_CASES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t Launch<real_t>::interp(int P, int ntiles, const real_t* grid, const Vec4<real_t>* rec, const int2* idx,
                                 const int* tile_off, const real_t* wcoef, const real_t* dwcoef, const Geom& g,
                                 Vec4<real_t> inv_alpha, double* phi, double* f, cudaStream_t s) {
    switch (P) {
#define X(p) case p: return interp_p<p>(ntiles, grid, rec, idx, tile_off, wcoef, dwcoef, g, inv_alpha, phi, f, s);
        PSWF_P_CASES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pswf
