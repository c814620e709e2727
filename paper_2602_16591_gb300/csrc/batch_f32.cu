// Fused float32 batch evaluation: the launches of batch.cuh's stage kernels and the batched FFTs.
#include <cufft.h>

#define PSWF_BATCH_KERNELS
#include "batch.cuh"
#include "launch.h"

namespace pswf {

namespace {

// radial degree buckets of the fused real-space kernel (float32 plans need at most ~16)
#define PSWF_BATCH_D_CASES(X) X(8) X(10) X(11) X(12) X(16)
#define PSWF_BATCH_P_CASES(X) \
    X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24)

template <int D>
cudaError_t short_d(const BatchRunF& r, cudaStream_t s) {
    auto kern = kb_short<D>;
    if (r.short_smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(r.short_smem));
        if (e != cudaSuccess) return e;
    }
    kern<<<r.total[kBShort], 32 * kShortWarps, r.short_smem, s>>>(
        r.sys, static_cast<const ShortParams<float, D>*>(r.kps), r.map + r.moff[kBShort]);
    return cudaGetLastError();
}

template <int P>
cudaError_t spread_p(const BatchRunF& r, cudaStream_t s) {
    auto kern = kb_spread<P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(r.spread_smem));
    if (e != cudaSuccess) return e;
    kern<<<r.total[kBSpread], spread_threads<P, kTile32>(), r.spread_smem, s>>>(
        r.sys, r.map + r.moff[kBSpread]);
    return cudaGetLastError();
}

template <int P>
cudaError_t interp_p(const BatchRunF& r, cudaStream_t s) {
    auto kern = kb_interp<P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(r.interp_smem));
    if (e != cudaSuccess) return e;
    kern<<<r.total[kBInterp], 32 * InterpCfg<float>::NWARP, r.interp_smem, s>>>(
        r.sys, r.map + r.moff[kBInterp], r.phi, r.f);
    return cudaGetLastError();
}

#define PSWF_TRY(call)                            \
    do {                                          \
        const cudaError_t e_ = (call);            \
        if (e_ != cudaSuccess) return e_;         \
    } while (0)

}  // namespace

bool batch_f32_supports(int P, int D) {
    bool pd = false, pp = false;
#define X(d) pd = pd || D == d;
    PSWF_BATCH_D_CASES(X)
#undef X
#define X(p) pp = pp || P == p;
    PSWF_BATCH_P_CASES(X)
#undef X
    return pd && pp;
}

cudaError_t batch_f32_run(const BatchRunF& r, cudaStream_t s, cudaStream_t s_short, cudaEvent_t fork,
                          cudaEvent_t join) {
    auto st = [&](int stage) { return r.map + r.moff[stage]; };
    // sort: zero the counters, count, scan, stable ranks, records
    kb_zero<<<r.total[kBZero], 256, 0, s>>>(r.sys, st(kBZero));
    kb_prep<<<r.total[kBPrep], 256, 0, s>>>(r.sys, st(kBPrep), r.x, r.rho);
    kb_scan<<<r.total[kBScan], 1024, 0, s>>>(r.sys, st(kBScan));
    kb_place<<<r.total[kBPlace], 256, 0, s>>>(r.sys, st(kBPlace));
    kb_rerank<<<r.total[kBRerank], 256, 0, s>>>(r.sys, st(kBRerank));
    kb_scatter<<<r.total[kBScatter], 256, 0, s>>>(r.sys, st(kBScatter), r.x, r.rho);
    PSWF_TRY(cudaGetLastError());
    // real-space sum on the second stream
    PSWF_TRY(cudaEventRecord(fork, s));
    PSWF_TRY(cudaStreamWaitEvent(s_short, fork, 0));
    cudaError_t e = cudaErrorInvalidValue;
    switch (r.D) {
#define X(d) case d: e = short_d<d>(r, s_short); break;
        PSWF_BATCH_D_CASES(X)
#undef X
        default: break;
    }
    PSWF_TRY(e);
    PSWF_TRY(cudaEventRecord(join, s_short));
    // Alg. 2: spread + halo, batched FFTs per grid size, scale, inverse FFTs, interpolation
    e = cudaErrorInvalidValue;
    switch (r.P) {
#define X(p) case p: e = spread_p<p>(r, s); break;
        PSWF_BATCH_P_CASES(X)
#undef X
        default: break;
    }
    PSWF_TRY(e);
    kb_halo<<<r.total[kBHalo], 256, 0, s>>>(r.sys, st(kBHalo));
    PSWF_TRY(cudaGetLastError());
    for (int k = 0; k < r.nfft; ++k) {
        const cufftHandle h = static_cast<cufftHandle>(r.ffts[k].handle_fwd);
        if (cufftSetStream(h, s) != CUFFT_SUCCESS || cufftExecR2C(h, r.ffts[k].a, reinterpret_cast<cufftComplex*>(r.ffts[k].spec)) != CUFFT_SUCCESS)
            return cudaErrorLaunchFailure;
    }
    kb_scale<<<r.total[kBScale], 256, 0, s>>>(r.sys, st(kBScale));
    PSWF_TRY(cudaGetLastError());
    for (int k = 0; k < r.nfft; ++k) {
        const cufftHandle h = static_cast<cufftHandle>(r.ffts[k].handle_inv);
        if (cufftSetStream(h, s) != CUFFT_SUCCESS || cufftExecC2R(h, reinterpret_cast<cufftComplex*>(r.ffts[k].spec), r.ffts[k].b) != CUFFT_SUCCESS)
            return cudaErrorLaunchFailure;
    }
    e = cudaErrorInvalidValue;
    switch (r.P) {
#define X(p) case p: e = interp_p<p>(r, s); break;
        PSWF_BATCH_P_CASES(X)
#undef X
        default: break;
    }
    PSWF_TRY(e);
    // join, then phi += real-space phi, F += real-space F, per-system energies
    PSWF_TRY(cudaStreamWaitEvent(s, join, 0));
    kb_combine<<<r.total[kBCombine], 256, 0, s>>>(r.sys, st(kBCombine), r.phi, r.f, r.rho);
    return cudaGetLastError();
}

}  // namespace pswf
