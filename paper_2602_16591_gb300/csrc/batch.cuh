// Fused evaluation of a batch of independent float32 systems: one launch per pipeline stage covers
// every system of the batch.  Each stage has a map from its blocks to {system, local block}; a block
// runs the single-system kernel body (the *_body functions of device.cuh) on that system's buffers with
// its local block index.  The FFTs
// run as one batched cuFFT plan per grid size.  Used for batches whose systems share the window
// support P (the P-templated spreading and interpolation bodies), with the radial polynomials padded
// to one degree bucket D.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"

namespace pswf {

// Everything one system's stage bodies need (device memory; one entry per system).  The radial
// polynomials of the real-space sum live in a separate ShortParams<float, D> array.
struct BatchSysF {
    Geom g;
    ScaleParams<float> sc;
    Vec4<float> inv_alpha;
    int* key_rank;
    int* perm;
    int* tile_cnt;
    int* tile_off;
    int* cell_cnt;
    int* cell_off;
    double* status;
    int* zeroed;
    Vec4<float>* sp_rec;
    int2* sp_idx;
    Vec4<float>* sr_rec;
    int2* sr_idx;
    Vec4<float>* sr_lo;
    float* scratch;
    float* grid_a;
    float* grid_b;
    float2* spec;
    const float* wcoef;
    const float* dwcoef;
    float* phi_sr;
    float* f_sr;
    double* epart;
    double* energy;
    int64_t off;        // first row of the system in the batch's x, rho, phi, F
    int zeroed_ints;    // 32-bit words of the per-evaluation zeroed block
    int ntiles, ncells, m3, nspec, rcap, degw, eblocks;
};

// Stages of the fused pipeline (segments of the block map).
enum BatchStage { kBZero, kBPrep, kBScan, kBPlace, kBRerank, kBScatter, kBShort, kBSpread, kBHalo, kBScale,
                  kBInterp, kBCombine, kBStages };

// Host side of a fused evaluation (batch_f32.cu): the batch's tables and buffers.
struct BatchFftF {
    int count;              // systems of this grid size
    int handle_fwd, handle_inv;   // cuFFT handles (cufftHandle)
    float* a;
    float* b;
    float2* spec;
};

struct BatchRunF {
    const BatchSysF* sys;   // device: one descriptor per system
    const void* kps;        // device: ShortParams<float, D>[nsys]
    const int2* map;        // device: block map of every stage, stage st at map + moff[st]
    const int* moff;        // host: offset of every stage's segment in map
    const int* total;       // host: blocks of every stage
    int nsys, P, D;
    size_t spread_smem, interp_smem, short_smem;
    const BatchFftF* ffts;  // host: one entry per grid size
    int nfft;
    const double* x;
    const double* rho;
    double* phi;
    double* f;
};

// Runs the fused pipeline: sort stages on s, then the real-space sum on s_short concurrently with
// Alg. 2 on s, joined on s before the combine stage.
cudaError_t batch_f32_run(const BatchRunF& r, cudaStream_t s, cudaStream_t s_short, cudaEvent_t fork,
                          cudaEvent_t join);
bool batch_f32_supports(int P, int D);

#ifdef PSWF_BATCH_KERNELS
// This block's system s and its block index inside that system's share of the launch: one entry per
// block of every stage ({system, local block}), read by all threads of the block (one broadcast load).
__device__ __forceinline__ void batch_block(const int2* __restrict__ map, int& s, int& local) {
    const int2 e = map[blockIdx.x];
    s = e.x;
    local = e.y;
}

__global__ void __launch_bounds__(256) kb_zero(const BatchSysF* __restrict__ sys, const int2* __restrict__ map) {
    int s, l;
    batch_block(map, s, l);
    const int i = l * 256 + threadIdx.x;
    if (i < sys[s].zeroed_ints) sys[s].zeroed[i] = 0;
}

__global__ void __launch_bounds__(256) kb_prep(const BatchSysF* __restrict__ sys, const int2* __restrict__ map, const double* __restrict__ x, const double* __restrict__ rho) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    k_prep_body<true>(l, x + 3 * b.off, rho + b.off, b.g, b.key_rank, b.tile_cnt, b.cell_cnt, b.status);
}

__global__ void __launch_bounds__(1024) kb_scan(const BatchSysF* __restrict__ sys, const int2* __restrict__ map) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    k_scan_body(l, b.tile_cnt, b.tile_off, b.ntiles, b.cell_cnt, b.cell_off, b.ncells);
}

__global__ void __launch_bounds__(256) kb_place(const BatchSysF* __restrict__ sys, const int2* __restrict__ map) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    k_place_body(l, b.key_rank, b.g.n, b.tile_off, b.cell_off, b.perm);
}

__global__ void __launch_bounds__(256) kb_rerank(const BatchSysF* __restrict__ sys, const int2* __restrict__ map) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    const int nb = (b.g.n + 255) / 256;   // the system's blocks: tiles first, then cells
    k_rerank_body(l % nb, l / nb, b.key_rank, b.g.n, b.tile_off, b.cell_off, b.perm);
}

__global__ void __launch_bounds__(256) kb_scatter(const BatchSysF* __restrict__ sys, const int2* __restrict__ map, const double* __restrict__ x, const double* __restrict__ rho) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    k_scatter_body<float>(l, x + 3 * b.off, rho + b.off, b.g, b.key_rank, b.tile_off, b.cell_off, b.sp_rec, b.sp_idx,
                          b.sr_rec, b.sr_idx, b.sr_lo, nullptr);
}

template <int D>
__global__ void __launch_bounds__(32 * kShortWarps, 6) kb_short(const BatchSysF* __restrict__ sys,
                                                                  const ShortParams<float, D>* __restrict__ kps,
                                                                  const int2* __restrict__ map) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    const ShortParams<float, D> kp = kps[s];   // the system's radial polynomials, in registers
    k_short_body<D>(l, b.sr_rec, b.sr_idx, b.sr_lo, b.cell_off, b.rcap, b.g, kp, b.phi_sr, b.f_sr);
}

template <int P>
__global__ void __launch_bounds__(spread_threads<P, kTile32>()) kb_spread(const BatchSysF* __restrict__ sys,
                                                                            const int2* __restrict__ map) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    k_spread_body<float, P>(l, b.sp_rec, b.sp_idx, b.tile_off, b.wcoef, b.degw,
                            SpreadChain{b.g.K, b.g.nt[1] * b.g.nt[2], b.ntiles}, b.scratch);
}

__global__ void __launch_bounds__(256) kb_halo(const BatchSysF* __restrict__ sys, const int2* __restrict__ map) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    k_halo_body<float, 0>(l, 0, b.scratch, b.tile_off, b.g, b.grid_a);
}

__global__ void __launch_bounds__(256) kb_scale(const BatchSysF* __restrict__ sys, const int2* __restrict__ map) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    k_scale_body<float, float2>(l, b.spec, b.sc);
}

template <int P>
__global__ void __launch_bounds__(32 * InterpCfg<float>::NWARP) kb_interp(const BatchSysF* __restrict__ sys, const int2* __restrict__ map, double* __restrict__ phi, double* __restrict__ f) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    k_interp_body<float, P>(l, b.grid_b, b.sp_rec, b.sp_idx, b.tile_off, b.wcoef, b.dwcoef, b.g, b.inv_alpha,
                            phi + b.off, f + 3 * b.off);
}

__global__ void __launch_bounds__(256) kb_combine(const BatchSysF* __restrict__ sys, const int2* __restrict__ map, double* __restrict__ phi, double* __restrict__ f,
                                                  const double* __restrict__ rho) {
    int s, l;
    batch_block(map, s, l);
    const BatchSysF& b = sys[s];
    k_combine_energy_body<float>(l, b.eblocks, phi + b.off, f + 3 * b.off, b.phi_sr, b.f_sr, rho + b.off, b.g.n,
                                 b.epart, reinterpret_cast<unsigned*>(b.status + 3), b.energy);
}
#endif  // PSWF_BATCH_KERNELS

}  // namespace pswf
