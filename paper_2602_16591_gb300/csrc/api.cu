// C ABI of the PSWF fast Ewald library: plan management, the evaluation pipeline and the
// host-side table entry points declared in include/pswf_ewald.h.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <future>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "batch.cuh"
#include "tc_spread.h"
#include "device.cuh"
#include "launch.h"
#include "planner.h"
#include "pswf_ewald.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

#define PSWF_CUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(EWALD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define PSWF_CUFFT(call)                                                                    \
    do {                                                                                    \
        cufftResult r_ = (call);                                                            \
        if (r_ != CUFFT_SUCCESS) return fail(EWALD_ECUFFT, std::string(#call) + " failed: " + std::to_string(r_)); \
    } while (0)

// Device memory of batch members comes from one pool owned by the batch (a few large cudaMalloc calls
// instead of ~35 per system); other plans allocate directly.  The pool in use is thread-local and set
// only while a batch creates its members.
struct DevicePool {
    std::vector<void*> chunks;
    char* cur = nullptr;
    size_t left = 0;
    cudaError_t alloc(void** p, size_t bytes) {
        bytes = (bytes + 255) & ~static_cast<size_t>(255);
        if (bytes > left) {
            const size_t sz = std::max(bytes, static_cast<size_t>(256) << 20);
            void* c = nullptr;
            const cudaError_t e = cudaMalloc(&c, sz);
            if (e != cudaSuccess) return e;
            chunks.push_back(c);
            cur = static_cast<char*>(c);
            left = sz;
        }
        *p = cur;
        cur += bytes;
        left -= bytes;
        return cudaSuccess;
    }
    ~DevicePool() {
        for (void* c : chunks) cudaFree(c);
    }
};
thread_local DevicePool* t_pool = nullptr;

cudaError_t dmalloc(void** p, size_t bytes) { return t_pool ? t_pool->alloc(p, bytes) : cudaMalloc(p, bytes); }
template <typename T>
cudaError_t dmalloc(T** p, size_t bytes) {
    return dmalloc(reinterpret_cast<void**>(p), bytes);
}

template <typename T>
int upload(T** dst, const std::vector<double>& src) {
    std::vector<T> tmp(src.begin(), src.end());
    if (dmalloc(dst, sizeof(T) * (tmp.empty() ? 1 : tmp.size())) != cudaSuccess)
        return fail(EWALD_ENOMEM, "cudaMalloc of a table failed");
    if (!tmp.empty() && cudaMemcpy(*dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(EWALD_ECUDA, "table upload failed");
    return EWALD_OK;
}

// Float-float table: the high parts of every coefficient followed by the low parts.
int upload_ff(float** dst, const std::vector<double>& src) {
    std::vector<float> tmp(2 * src.size());
    for (size_t i = 0; i < src.size(); ++i) {
        tmp[i] = static_cast<float>(src[i]);
        tmp[src.size() + i] = static_cast<float>(src[i] - static_cast<double>(tmp[i]));
    }
    if (dmalloc(dst, sizeof(float) * (tmp.empty() ? 1 : tmp.size())) != cudaSuccess)
        return fail(EWALD_ENOMEM, "cudaMalloc of a table failed");
    if (!tmp.empty() && cudaMemcpy(*dst, tmp.data(), sizeof(float) * tmp.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(EWALD_ECUDA, "table upload failed");
    return EWALD_OK;
}

// Smallest kf in [1, deg_w] such that a float32 Horner pass over the window terms k >= kf errs by at
// most a quarter of the fit tolerance: 2^-23 (deg_w - kf + 1) max_a sum_{k >= kf} |c_ak| (|z| <= 1),
// for the window (scale 1) and its derivative (scale max |psi'| / psi(0)).
int ff_split_index(const pswf::HostPlan& hp) {
    const int P = hp.p.P, d = hp.p.deg_w;
    double dscale = 0;
    for (int a = 0; a < P; ++a) dscale = std::max(dscale, std::fabs(hp.dwc[a * (d + 1)]));
    auto tail_ok = [&](const std::vector<double>& c, int kf, double scale) {
        double mx = 0;
        for (int a = 0; a < P; ++a) {
            double t = 0;
            for (int k = kf; k <= d; ++k) t += std::fabs(c[a * (d + 1) + k]);
            mx = std::max(mx, t);
        }
        return std::ldexp(mx * (d - kf + 1), -23) <= 0.25 * hp.p.fit_tol * scale;
    };
    for (int kf = 1; kf <= d; ++kf)
        if (tail_ok(hp.wc, kf, 1.0) && tail_ok(hp.dwc, kf, std::max(dscale, 1.0))) return kf;
    return d;
}

// Smallest kr such that float32 Horner steps over the radial terms k >= kr err by at most
// 2.5 fit_tol max|f| (= tol_plan / 20 of the polynomial's scale; the pair errors enter the potential with
// random signs): 2^-23 (deg_r - kr + 1) sum_{k >= kr} |c_k| (|u| <= 1).  deg_r + 1: all float-float.
int ff_radial_split(const pswf::HostPlan& hp) {
    const int d = hp.p.deg_r;
    auto smax = [&](const std::vector<double>& c) {
        double m = 0;
        for (int i = 0; i <= 200; ++i) m = std::max(m, std::fabs(pswf::horner(c.data(), d, -1.0 + i / 100.0)));
        return m;
    };
    const double s1 = smax(hp.p1c), s2 = smax(hp.qc);
    auto ok = [&](const std::vector<double>& c, int kr, double sc) {
        double t = 0;
        for (int k = kr; k <= d; ++k) t += std::fabs(c[k]);
        return std::ldexp(t * (d - kr + 1), -23) <= 2.5 * hp.p.fit_tol * sc;
    };
    for (int kr = 1; kr <= d; ++kr)
        if (ok(hp.p1c, kr, s1) && ok(hp.qc, kr, s2)) return kr;
    return d + 1;
}

}  // namespace

namespace pswf {
// Lets other translation units of the library set the message ewald_last_error() returns.
void record_error(const std::string& msg) { g_last_error = msg; }
}  // namespace pswf

namespace {

// cuFFT plans are shared process-wide by (device, m, type): creating them dominates the setup of small
// plans, and batches hold many systems of the same grid size.  A shared handle is used only under
// g_fft_mu: each exec first sets the calling plan's stream and its own work area (the work area
// pointer is fixed into the launched kernels at exec time, also during graph capture).
struct FftCache {
    std::mutex mu;
    std::map<std::tuple<int, int, int, int, int>, std::pair<cufftHandle, size_t>> plans;   // -> (handle, work)
};
FftCache& fft_cache() {
    static FftCache* c = new FftCache();   // never destroyed: handles outlive static teardown order
    return *c;
}

int shared_fft(int device, const int* m, cufftType type, cufftHandle* h, size_t* work) {
    FftCache& c = fft_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    const auto key = std::make_tuple(device, m[0], m[1], m[2], static_cast<int>(type));
    auto it = c.plans.find(key);
    if (it == c.plans.end()) {
        cufftHandle nh = 0;
        size_t ws = 0;
        if (cufftCreate(&nh) != CUFFT_SUCCESS) return fail(EWALD_ECUFFT, "cufftCreate failed");
        if (cufftSetAutoAllocation(nh, 0) != CUFFT_SUCCESS ||
            cufftMakePlan3d(nh, m[0], m[1], m[2], type, &ws) != CUFFT_SUCCESS) {
            cufftDestroy(nh);
            return fail(EWALD_ECUFFT, "cufftMakePlan3d failed for a " + std::to_string(m[0]) + " x " +
                                          std::to_string(m[1]) + " x " + std::to_string(m[2]) + " grid");
        }
        it = c.plans.emplace(key, std::make_pair(nh, ws)).first;
    }
    *h = it->second.first;
    *work = it->second.second;
    return EWALD_OK;
}

}  // namespace

struct ewald_plan_s {
    pswf::HostPlan hp;
    pswf::Geom g{};
    int device = 0;
    bool fp64 = true;   // grid, FFT and scaling in float64 (EWALD_FP64 and EWALD_FLOATFLOAT plans)
    bool ff = false;    // float-float particle kernels (EWALD_FLOATFLOAT)
    int ff_kf = 1;      // window polynomial terms k >= ff_kf are summed in float32 (float-float plans)
    int ff_kr = 1;      // radial polynomial terms k >= ff_kr likewise
    int ntiles = 0, ncells = 0, epart_blocks = 0;
    size_t m3 = 0, nspec = 0;   // grid points, half-spectrum modes
    // workspace
    int* key_rank = nullptr;
    int* perm = nullptr;       // bin lists of the stable counting sort (tile order, then cell order)
    int* tile_cnt = nullptr;
    int* tile_off = nullptr;
    int* cell_cnt = nullptr;
    int* cell_off = nullptr;
    void* sp_rec = nullptr;
    int2* sp_idx = nullptr;
    void* sr_rec = nullptr;
    int2* sr_idx = nullptr;
    void* sr_lo = nullptr;   // float32 plans: float-float residue of the local coordinates
    float4* sr_f32 = nullptr;  // float64 plans: float32 copy of the local coordinates (cutoff pre-test)
    int* sr_cz = nullptr;      // float-float plans: z cell index of every cell-sorted record
    void* grid_ff = nullptr;   // float-float plans: the interpolation grid as {hi, lo} float pairs
    int4* sr_cols = nullptr;   // real-space columns {dx, dy, dzmax, 0} with box distance < rc
    int* scan_tmp = nullptr;   // multi-block scan: block sums and offsets of both segments (long arrays only)
    int* tc_err = nullptr;     // tensor-core spreading: set when an MMA completion wait ran out (zeroed block)
    bool tc_spread = false;
    int scan_nb0 = 0, scan_nb1 = 0;
    int n_cols = 0;
    int sr_rcap = 0;           // bound on the contiguous source ranges of one neighbourhood
    void* scratch = nullptr;
    void* grid_a = nullptr;
    void* grid_b = nullptr;
    void* spec = nullptr;
    bool pooled_grids = false;   // grid_a, grid_b, spec belong to a fused batch's pool (not freed here)
    bool pooled = false;         // every device buffer comes from a batch's DevicePool (not freed here)
    std::unique_ptr<DevicePool> pool;   // batch plans: the members' device memory
    void* wcoef = nullptr;
    void* dwcoef = nullptr;
    void* p1c = nullptr;
    void* qc = nullptr;
    void* iw = nullptr;
    void* mtab = nullptr;
    void* gcoef = nullptr;   // cuboid boxes: mollifier transform polynomial (scaling step)
    double* phi_int = nullptr;
    double* f_int = nullptr;
    double* status = nullptr;
    void* zeroed = nullptr;      // status words, tile and cell counters: one block, cleared by one memset
    size_t zeroed_bytes = 0;
    double* epart = nullptr;
    double* energy_d = nullptr;
    double* x_stage = nullptr;
    double* rho_stage = nullptr;
    double* status_h = nullptr;   // pinned
    cufftHandle fwd = 0, inv = 0;   // shared (fft_cache), not owned
    void* fft_work = nullptr;        // this plan's cuFFT work area (forward and inverse run in sequence)
    // the real-space sum runs on its own stream, concurrently with spread -> FFT -> interpolation
    // (Alg. 2 on a high-priority stream so its short kernels are not starved by the real-space blocks)
    cudaStream_t s_short = nullptr, s_alg2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    double* phi_sr = nullptr;   // real-space potential and forces, merged by k_combine_energy
    double* f_sr = nullptr;
    // batch plans (ewald_plan_batch_create): one plan per system, evaluated as one captured graph
    bool is_batch = false;
    std::vector<ewald_plan_s*> members;
    std::vector<int64_t> offsets;              // prefix sums of the systems' particle counts
    std::vector<cudaStream_t> bstreams;         // per-system streams of the capture (fork / join)
    std::vector<cudaEvent_t> bevents;
    cudaEvent_t bstart = nullptr;
    cudaStream_t bcap = nullptr;                // capture origin
    cudaGraphExec_t bexec = nullptr;
    const void* bkey[4] = {nullptr, nullptr, nullptr, nullptr};   // buffers the graph was captured with
    double* bout_d = nullptr;                   // per system {sum rho, sum |rho|, non-finite, energy}
    double* bout_h = nullptr;                   // pinned
    const double** bsrc_d = nullptr;            // per system {status, energy} device pointers
    // fused float32 batches (batch.cuh): one launch per stage over all systems, cuFFT batched per grid size
    bool fused = false;
    int bD = 0, bP = 0;                          // radial degree bucket and window support of the batch
    void* bsys_d = nullptr;                      // BatchSysF[nsys]
    void* bkp_d = nullptr;                       // ShortParams<float, bD>[nsys]
    int2* bmap_d = nullptr;                      // {system, local block} for every block of every stage
    std::vector<int> btotal, bmoff;              // blocks of every stage, offset of its segment in bmap_d
    size_t bspread_smem = 0, binterp_smem = 0, bshort_smem = 0;
    struct FftGroup {
        int m = 0, count = 0;
        float* a = nullptr;
        float* b = nullptr;
        float2* spec = nullptr;
        cufftHandle fwd = 0, inv = 0;
    };
    std::vector<FftGroup> fgroups;
    cudaStream_t bs_short = nullptr;
    cudaEvent_t bfork = nullptr, bjoin = nullptr;
    bool profiling = false;
    bool serial = false;   // profiling mode 2: real-space sum and Alg. 2 serialised on the caller's stream
    std::vector<std::vector<cudaEvent_t>> prof;   // begin/end event of every stage per recorded evaluation
    std::vector<cudaEvent_t>* cur = nullptr;

    void mark(int k, bool end, cudaStream_t s) {
        if (cur) cudaEventRecord((*cur)[2 * k + (end ? 1 : 0)], s);
    }
    void clear_prof() {
        for (auto& v : prof)
            for (cudaEvent_t e : v) cudaEventDestroy(e);
        prof.clear();
        cur = nullptr;
    }

    ~ewald_plan_s() {
        void* bufs[] = {key_rank, perm, zeroed, tile_off, cell_off, sp_rec, sp_idx, sr_rec, sr_idx, sr_lo, sr_f32, sr_cz, grid_ff, sr_cols, scan_tmp, scratch,
                        pooled_grids ? nullptr : grid_a, pooled_grids ? nullptr : grid_b, pooled_grids ? nullptr : spec,
                        wcoef, dwcoef, p1c, qc, iw, mtab, gcoef, phi_int, f_int, epart, energy_d, x_stage, rho_stage};
        for (void* b : bufs)
            if (b && !pooled) cudaFree(b);
        if (status_h) cudaFreeHost(status_h);
        clear_prof();
        if (phi_sr && !pooled) cudaFree(phi_sr);
        if (f_sr && !pooled) cudaFree(f_sr);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (ev_join2) cudaEventDestroy(ev_join2);
        if (s_short) cudaStreamDestroy(s_short);
        if (s_alg2) cudaStreamDestroy(s_alg2);
        if (fft_work && !pooled) cudaFree(fft_work);
        for (ewald_plan_s* m : members) delete m;
        for (cudaStream_t st : bstreams)
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t e : bevents)
            if (e) cudaEventDestroy(e);
        if (bstart) cudaEventDestroy(bstart);
        if (bcap) cudaStreamDestroy(bcap);
        if (bexec) cudaGraphExecDestroy(bexec);
        if (bout_d) cudaFree(bout_d);
        if (bout_h) cudaFreeHost(bout_h);
        if (bsrc_d) cudaFree(bsrc_d);
        if (bsys_d) cudaFree(bsys_d);
        if (bkp_d) cudaFree(bkp_d);
        if (bmap_d) cudaFree(bmap_d);
        for (auto& fg : fgroups) {
            if (fg.fwd) cufftDestroy(fg.fwd);
            if (fg.inv) cufftDestroy(fg.inv);
            if (fg.a) cudaFree(fg.a);
            if (fg.b) cudaFree(fg.b);
            if (fg.spec) cudaFree(fg.spec);
        }
        if (bs_short) cudaStreamDestroy(bs_short);
        if (bfork) cudaEventDestroy(bfork);
        if (bjoin) cudaEventDestroy(bjoin);
    }
};

namespace {

template <typename real>
pswf::ScaleParams<real> scale_params(ewald_plan p) {
    pswf::ScaleParams<real> sp{};
    const ewald_params& q = p->hp.p;
    for (int d = 0; d < 3; ++d) {
        sp.m[d] = q.grid[d];
        sp.w2[d] = static_cast<real>((2.0 * 3.14159265358979323846 / q.box[d]) * (2.0 * 3.14159265358979323846 / q.box[d]));
    }
    sp.cube = q.deg_g == 0;
    sp.degg = q.deg_g;
    sp.tscale = static_cast<real>((q.rc / q.cs) * (q.rc / q.cs));
    sp.four_pi_over_V = static_cast<real>(4.0 * 3.14159265358979323846 / (q.box[0] * q.box[1] * q.box[2]));
    sp.iw = static_cast<const real*>(p->iw);
    sp.mtab = static_cast<const real*>(p->mtab);
    sp.gc = static_cast<const real*>(p->gcoef);
    return sp;
}

// Runs a shared cuFFT plan on stream s with plan p's work area.
template <class F>
int fft_exec(ewald_plan p, cufftHandle h, cudaStream_t s, F exec) {
    std::lock_guard<std::mutex> lk(fft_cache().mu);
    PSWF_CUFFT(cufftSetStream(h, s));
    PSWF_CUFFT(cufftSetWorkArea(h, p->fft_work));
    PSWF_CUFFT(exec());
    return EWALD_OK;
}

template <typename real, int D>
cudaError_t launch_short_d(ewald_plan p, const pswf::Vec4<real>* sr_rec, const pswf::Vec4<real>* sr_lo, double* phi,
                           double* f, cudaStream_t s) {
    const pswf::Geom& g = p->g;
    pswf::ShortParams<real, D> kp{};
    const auto& c1 = p->hp.p1c;
    const auto& c2 = p->hp.qc;
    for (int k = 0; k <= D; ++k) {
        kp.p1[k] = static_cast<real>(k < static_cast<int>(c1.size()) ? c1[k] : 0.0);
        kp.q[k] = static_cast<real>(k < static_cast<int>(c2.size()) ? c2[k] : 0.0);
    }
    kp.rc2 = static_cast<real>(g.rc * g.rc);
    kp.two_over_rc2 = static_cast<real>(2.0 / (g.rc * g.rc));
    kp.rc2f = static_cast<float>(g.rc * g.rc * (1.0 + 1e-4));
    const int ncells = g.ncell[0] * g.ncell[1] * g.ncell[2];
    const size_t smem = sizeof(real) == 4 ? pswf::short_dyn_smem_f32(p->sr_rcap) : pswf::short_dyn_smem(p->sr_rcap);
    const int blocks = (ncells + pswf::kShortWarps - 1) / pswf::kShortWarps;
    // float32 pairs are cheap: one target at a time, full-warp masked pairs over the target's own
    // neighbourhood; float64 pairs: the two-phase (queued) kernel over cells
    if constexpr (sizeof(real) == 4) {
        const int per_block = pswf::kShortWarps * pswf::kShortTPW;
        pswf::k_short<D><<<(g.n + per_block - 1) / per_block, 32 * pswf::kShortWarps, smem, s>>>(
            sr_rec, p->sr_idx, sr_lo, p->cell_off, p->sr_rcap, g, kp,
            reinterpret_cast<float*>(phi), reinterpret_cast<float*>(f));   // float results in the float64 buffers
    } else {
        pswf::k_short_q<D><<<blocks, 32 * pswf::kShortWarps, smem, s>>>(
            sr_rec, p->sr_idx, p->sr_f32, p->cell_off, p->sr_cols, p->n_cols, p->sr_rcap, g, kp, phi, f);
    }
    return cudaGetLastError();
}

// Radial polynomial degrees are rounded up to a bucket; the padding coefficients are zero.
template <typename real>
cudaError_t launch_short(ewald_plan p, const pswf::Vec4<real>* sr_rec, const pswf::Vec4<real>* sr_lo, double* phi,
                         double* f, cudaStream_t s) {
    const int d = p->g.degr;
    if (d <= 8) return launch_short_d<real, 8>(p, sr_rec, sr_lo, phi, f, s);
    if (d <= 10) return launch_short_d<real, 10>(p, sr_rec, sr_lo, phi, f, s);
    if (d == 11) return launch_short_d<real, 11>(p, sr_rec, sr_lo, phi, f, s);   // tol ~1e-6
    if (d <= 12) return launch_short_d<real, 12>(p, sr_rec, sr_lo, phi, f, s);
    if (d <= 16) return launch_short_d<real, 16>(p, sr_rec, sr_lo, phi, f, s);
    if (d <= 20) return launch_short_d<real, 20>(p, sr_rec, sr_lo, phi, f, s);
    if (d <= 24) return launch_short_d<real, 24>(p, sr_rec, sr_lo, phi, f, s);
    if (d <= 32) return launch_short_d<real, 32>(p, sr_rec, sr_lo, phi, f, s);
    if (d <= 44) return launch_short_d<real, 44>(p, sr_rec, sr_lo, phi, f, s);
    return launch_short_d<real, 60>(p, sr_rec, sr_lo, phi, f, s);
}

// Input-order ranks inside every tile and cell (k_place, k_rerank), after the counting scan.
cudaError_t stable_ranks(ewald_plan p, cudaStream_t s) {
    const int n = p->g.n, tb = 256, nb = (n + tb - 1) / tb;
    pswf::k_place<<<nb, tb, 0, s>>>(p->key_rank, n, p->tile_off, p->cell_off, p->perm);
    pswf::k_rerank<<<dim3(nb, 2), tb, 0, s>>>(p->key_rank, n, p->tile_off, p->cell_off, p->perm);
    return cudaGetLastError();
}

// Counting-sort offsets of the tiles and cells: one block per segment for short arrays; beyond
// kScanMulti counters the multi-block form (a single block would walk the chunks one after another).
constexpr int kScanMulti = 4 * pswf::kScanChunk;
constexpr int kNumSMs = 152;   // GB300 streaming multiprocessors
inline int round4(int v) { return (v + 3) & ~3; }   // int4 alignment of the sub-arrays of scan_tmp
size_t scan_tmp_ints(int nb0, int nb1) { return round4(nb0) + round4(nb1) + round4(nb0 + 1) + round4(nb1 + 1); }

cudaError_t launch_scan(ewald_plan p, cudaStream_t s) {
    if (!p->scan_tmp) {
        pswf::k_scan<<<2, 1024, 0, s>>>(p->tile_cnt, p->tile_off, p->ntiles, p->cell_cnt, p->cell_off, p->ncells);
        return cudaGetLastError();
    }
    const int nb0 = p->scan_nb0, nb1 = p->scan_nb1;
    int* bsum0 = p->scan_tmp;
    int* bsum1 = bsum0 + round4(nb0);
    int* boff0 = bsum1 + round4(nb1);
    int* boff1 = boff0 + round4(nb0 + 1);
    pswf::k_scan_sums<<<nb0 + nb1, 1024, 0, s>>>(p->tile_cnt, p->ntiles, nb0, p->cell_cnt, p->ncells, bsum0, bsum1);
    pswf::k_scan<<<2, 1024, 0, s>>>(bsum0, boff0, nb0, bsum1, boff1, nb1);
    pswf::k_scan_apply<<<nb0 + nb1, 1024, 0, s>>>(p->tile_cnt, p->tile_off, p->ntiles, nb0, p->cell_cnt, p->cell_off,
                                                  p->ncells, boff0, boff1);
    return cudaGetLastError();
}

template <typename real, typename cplx>
int run_pipeline(ewald_plan p, const double* x, const double* rho, double* phi, double* f, cudaStream_t s) {
    using pswf::Vec4;
    const pswf::Geom& g = p->g;
    const int n = g.n;
    p->mark(0, false, s);
    PSWF_CUDA(cudaMemsetAsync(p->zeroed, 0, p->zeroed_bytes, s));
    const int tb = 256, nb = (n + tb - 1) / tb;
    pswf::k_prep<std::is_same<real, float>::value><<<nb, tb, 0, s>>>(x, rho, g, p->key_rank, p->tile_cnt, p->cell_cnt, p->status);
    PSWF_CUDA(cudaGetLastError());
    PSWF_CUDA(launch_scan(p, s));
    PSWF_CUDA(stable_ranks(p, s));
    auto* sp_rec = static_cast<Vec4<real>*>(p->sp_rec);
    auto* sr_rec = static_cast<Vec4<real>*>(p->sr_rec);
    auto* sr_lo = static_cast<Vec4<real>*>(p->sr_lo);
    pswf::k_scatter<real><<<nb, tb, 0, s>>>(x, rho, g, p->key_rank, p->tile_off, p->cell_off, sp_rec, p->sp_idx,
                                            sr_rec, p->sr_idx, sr_lo, p->sr_f32);
    PSWF_CUDA(cudaGetLastError());
    p->mark(0, true, s);
    // real-space sum on the second stream, concurrent with Alg. 2
    // the real-space sum and Alg. 2 run concurrently on two streams, or one after the other on the
    // caller's stream when profiling in serial mode (stage times without overlap)
    const cudaStream_t s_short = p->serial ? s : p->s_short, s_alg2 = p->serial ? s : p->s_alg2;
    PSWF_CUDA(cudaEventRecord(p->ev_fork, s));
    PSWF_CUDA(cudaStreamWaitEvent(s_short, p->ev_fork, 0));
    p->mark(7, false, s_short);
    PSWF_CUDA(launch_short<real>(p, sr_rec, sr_lo, p->phi_sr, p->f_sr, s_short));
    p->mark(7, true, s_short);
    PSWF_CUDA(cudaEventRecord(p->ev_join, s_short));
    // Alg. 2 on the high-priority stream
    const cudaStream_t caller = s;
    PSWF_CUDA(cudaStreamWaitEvent(s_alg2, p->ev_fork, 0));
    s = s_alg2;
    // Alg. 2 step 1
    p->mark(1, false, s);
    if constexpr (sizeof(real) == 4) {
        if (p->tc_spread) {
            PSWF_CUDA(pswf::launch_spread_tc(g.P, p->ntiles, sp_rec, p->sp_idx, p->tile_off,
                                             static_cast<const float*>(p->wcoef), g.degw,
                                             pswf::SpreadChain{g.K, g.nt[1] * g.nt[2], p->ntiles},
                                             static_cast<float*>(p->scratch), p->tc_err, s));
        }
    }
    if (!p->tc_spread)
        PSWF_CUDA(pswf::Launch<real>::spread(g.P, p->ntiles, sp_rec, p->sp_idx, p->tile_off,
                                             static_cast<const real*>(p->wcoef), g.degw,
                                             pswf::SpreadChain{g.K, g.nt[1] * g.nt[2], p->ntiles},
                                             static_cast<real*>(p->scratch), s));
    p->mark(1, true, s);
    p->mark(2, false, s);
    const int mm = static_cast<int>(p->m3);
    {
        const int ni = (g.T + g.P - 1 + g.T - 1) / g.T;   // overlapping slabs per axis
        const auto* sc = static_cast<const real*>(p->scratch);
        auto* ga = static_cast<real*>(p->grid_a);
        // float32 plans (tile edge 8): 32 x 8 blocks over (z, y), grid (m_z / 32, m_y / 8, m_x); otherwise 1-D
        const dim3 hrow((g.m[2] + 31) / 32, (g.m[1] + 7) / 8, g.m[0]), hblk(32, 8);
        const int hb = (mm + 255) / 256;
        const bool rows = sizeof(real) == 4 && g.T == pswf::kTile32;
        if (rows && ni <= 2) pswf::k_halo<real, 2><<<hrow, hblk, 0, s>>>(sc, p->tile_off, g, ga);
        else if (rows && ni == 3) pswf::k_halo<real, 3><<<hrow, hblk, 0, s>>>(sc, p->tile_off, g, ga);
        else if (rows && ni == 4) pswf::k_halo<real, 4><<<hrow, hblk, 0, s>>>(sc, p->tile_off, g, ga);
        else pswf::k_halo<real, 0><<<hb, 256, 0, s>>>(sc, p->tile_off, g, ga);
    }
    PSWF_CUDA(cudaGetLastError());
    // Alg. 2 steps 2-4
    p->mark(2, true, s);
    p->mark(3, false, s);
    int frc;
    if constexpr (sizeof(real) == 8) {
        frc = fft_exec(p, p->fwd, s, [&] {
            return cufftExecD2Z(p->fwd, static_cast<cufftDoubleReal*>(p->grid_a), static_cast<cufftDoubleComplex*>(p->spec));
        });
    } else {
        frc = fft_exec(p, p->fwd, s, [&] {
            return cufftExecR2C(p->fwd, static_cast<cufftReal*>(p->grid_a), static_cast<cufftComplex*>(p->spec));
        });
    }
    if (frc) return frc;
    p->mark(3, true, s);
    p->mark(4, false, s);
    const int ns = static_cast<int>(p->nspec);
    pswf::k_scale<real, cplx><<<(ns + 255) / 256, 256, 0, s>>>(static_cast<cplx*>(p->spec), scale_params<real>(p));
    PSWF_CUDA(cudaGetLastError());
    p->mark(4, true, s);
    p->mark(5, false, s);
    if constexpr (sizeof(real) == 8) {
        frc = fft_exec(p, p->inv, s, [&] {
            return cufftExecZ2D(p->inv, static_cast<cufftDoubleComplex*>(p->spec), static_cast<cufftDoubleReal*>(p->grid_b));
        });
    } else {
        frc = fft_exec(p, p->inv, s, [&] {
            return cufftExecC2R(p->inv, static_cast<cufftComplex*>(p->spec), static_cast<cufftReal*>(p->grid_b));
        });
    }
    if (frc) return frc;
    p->mark(5, true, s);
    p->mark(6, false, s);
    // Alg. 2 step 5 + self term + forces
    // 1/alpha_d = 2 m_d / (P L_d) per axis (alpha_d = P h_d / 2; equal for cubes)
    const pswf::Vec4<real> inv_alpha{static_cast<real>(2.0 * g.m[0] / (g.P * g.L[0])),
                                     static_cast<real>(2.0 * g.m[1] / (g.P * g.L[1])),
                                     static_cast<real>(2.0 * g.m[2] / (g.P * g.L[2])), real(0)};
    PSWF_CUDA(pswf::Launch<real>::interp(g.P, p->ntiles, static_cast<const real*>(p->grid_b), sp_rec, p->sp_idx,
                                         p->tile_off, static_cast<const real*>(p->wcoef),
                                         static_cast<const real*>(p->dwcoef), g, inv_alpha, phi, f, s));
    p->mark(6, true, s);
    // join both branches on the caller's stream, merge the real-space sum into phi and F, energy
    PSWF_CUDA(cudaEventRecord(p->ev_join2, s));
    s = caller;
    PSWF_CUDA(cudaStreamWaitEvent(s, p->ev_join, 0));
    PSWF_CUDA(cudaStreamWaitEvent(s, p->ev_join2, 0));
    p->mark(8, false, s);
    pswf::k_combine_energy<real><<<p->epart_blocks, 256, 0, s>>>(phi, f, reinterpret_cast<const real*>(p->phi_sr),
                                                                 reinterpret_cast<const real*>(p->f_sr), rho, n, p->epart,
                                                           reinterpret_cast<unsigned*>(p->status + 3), p->energy_d);
    PSWF_CUDA(cudaGetLastError());
    p->mark(8, true, s);
    return EWALD_OK;
}

// Float-float plans: same stages and streams as run_pipeline; particle kernels from LaunchFF, float64
// grid, cuFFT D2Z/Z2D and k_scale.
int run_pipeline_ff(ewald_plan p, const double* x, const double* rho, double* phi, double* f, cudaStream_t s) {
    using pswf::LaunchFF;
    const pswf::Geom& g = p->g;
    const int n = g.n;
    const size_t nn = static_cast<size_t>(n);
    p->mark(0, false, s);
    PSWF_CUDA(cudaMemsetAsync(p->zeroed, 0, p->zeroed_bytes, s));
    const int tb = 256, nb = (n + tb - 1) / tb;
    pswf::k_prep<false><<<nb, tb, 0, s>>>(x, rho, g, p->key_rank, p->tile_cnt, p->cell_cnt, p->status);
    PSWF_CUDA(cudaGetLastError());
    PSWF_CUDA(launch_scan(p, s));
    PSWF_CUDA(stable_ranks(p, s));
    auto* sp_h = static_cast<float4*>(p->sp_rec);
    auto* sp_l = sp_h + nn;
    auto* sr_h = static_cast<float4*>(p->sr_rec);
    auto* sr_l = sr_h + nn;
    PSWF_CUDA(LaunchFF::scatter(x, rho, g, p->key_rank, p->tile_off, p->cell_off, sp_h, sp_l, p->sp_idx, sr_h, sr_l,
                                p->sr_idx, p->sr_cz, s));
    p->mark(0, true, s);
    // the real-space sum and Alg. 2 run concurrently on two streams, or one after the other on the
    // caller's stream when profiling in serial mode (stage times without overlap)
    const cudaStream_t s_short = p->serial ? s : p->s_short, s_alg2 = p->serial ? s : p->s_alg2;
    PSWF_CUDA(cudaEventRecord(p->ev_fork, s));
    PSWF_CUDA(cudaStreamWaitEvent(s_short, p->ev_fork, 0));
    p->mark(7, false, s_short);
    PSWF_CUDA(LaunchFF::short_range(g, sr_h, sr_l, p->sr_idx, p->sr_cz, p->cell_off, p->sr_cols, p->n_cols,
                                    p->sr_rcap, p->hp.p1c.data(), p->hp.qc.data(), p->ff_kr, p->phi_sr, p->f_sr,
                                    s_short));
    p->mark(7, true, s_short);
    PSWF_CUDA(cudaEventRecord(p->ev_join, s_short));
    const cudaStream_t caller = s;
    PSWF_CUDA(cudaStreamWaitEvent(s_alg2, p->ev_fork, 0));
    s = s_alg2;
    const auto* wc = static_cast<const float*>(p->wcoef);
    const auto* dwc = static_cast<const float*>(p->dwcoef);
    p->mark(1, false, s);
    PSWF_CUDA(LaunchFF::spread(p->ntiles, g, sp_h, sp_l, p->sp_idx, p->tile_off, wc, p->ff_kf,
                               static_cast<float2*>(p->scratch), s));
    p->mark(1, true, s);
    p->mark(2, false, s);
    PSWF_CUDA(LaunchFF::halo(static_cast<const float2*>(p->scratch), p->tile_off, g, static_cast<double*>(p->grid_a), s));
    p->mark(2, true, s);
    p->mark(3, false, s);
    int frc = fft_exec(p, p->fwd, s, [&] {
        return cufftExecD2Z(p->fwd, static_cast<cufftDoubleReal*>(p->grid_a), static_cast<cufftDoubleComplex*>(p->spec));
    });
    if (frc) return frc;
    p->mark(3, true, s);
    p->mark(4, false, s);
    const int ns = static_cast<int>(p->nspec);
    pswf::k_scale<double, cufftDoubleComplex><<<(ns + 255) / 256, 256, 0, s>>>(
        static_cast<cufftDoubleComplex*>(p->spec), scale_params<double>(p));
    PSWF_CUDA(cudaGetLastError());
    p->mark(4, true, s);
    p->mark(5, false, s);
    frc = fft_exec(p, p->inv, s, [&] {
        return cufftExecZ2D(p->inv, static_cast<cufftDoubleComplex*>(p->spec), static_cast<cufftDoubleReal*>(p->grid_b));
    });
    if (frc) return frc;
    const size_t m3 = p->m3;
    PSWF_CUDA(LaunchFF::to_ff(static_cast<const double*>(p->grid_b), m3, static_cast<float2*>(p->grid_ff), s));
    p->mark(5, true, s);
    p->mark(6, false, s);
    const double inv_alpha[3] = {2.0 * g.m[0] / (g.P * g.L[0]), 2.0 * g.m[1] / (g.P * g.L[1]),
                                 2.0 * g.m[2] / (g.P * g.L[2])};   // 1/alpha_d per axis
    PSWF_CUDA(LaunchFF::interp(p->ntiles, g, static_cast<const float2*>(p->grid_ff), sp_h, sp_l, p->sp_idx,
                               p->tile_off, wc, dwc, p->ff_kf, inv_alpha, phi, f, s));
    p->mark(6, true, s);
    PSWF_CUDA(cudaEventRecord(p->ev_join2, s));
    s = caller;
    PSWF_CUDA(cudaStreamWaitEvent(s, p->ev_join, 0));
    PSWF_CUDA(cudaStreamWaitEvent(s, p->ev_join2, 0));
    p->mark(8, false, s);
    pswf::k_combine_energy<double><<<p->epart_blocks, 256, 0, s>>>(phi, f, p->phi_sr, p->f_sr, rho, n, p->epart,
                                                           reinterpret_cast<unsigned*>(p->status + 3), p->energy_d);
    PSWF_CUDA(cudaGetLastError());
    p->mark(8, true, s);
    return EWALD_OK;
}

int eval_device(ewald_plan p, const double* x, const double* rho, double* phi, double* force, cudaStream_t s) {
    p->cur = nullptr;
    if (p->profiling) {
        std::vector<cudaEvent_t> ev(2 * EWALD_NSTAGES);
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(EWALD_ECUDA, "cudaEventCreate failed");
        p->prof.push_back(ev);
        p->cur = &p->prof.back();
    }
    double* phi_d = phi ? phi : p->phi_int;
    double* f_d = force ? force : p->f_int;
    if (p->ff) return run_pipeline_ff(p, x, rho, phi_d, f_d, s);
    if (p->fp64) return run_pipeline<double, cufftDoubleComplex>(p, x, rho, phi_d, f_d, s);
    return run_pipeline<float, cufftComplex>(p, x, rho, phi_d, f_d, s);
}

int read_status(ewald_plan p, cudaStream_t s, double* energy) {
    PSWF_CUDA(cudaMemcpyAsync(p->status_h, p->status, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    if (energy) PSWF_CUDA(cudaMemcpyAsync(p->status_h + 3, p->energy_d, sizeof(double), cudaMemcpyDeviceToHost, s));
    int* tc_err_h = reinterpret_cast<int*>(p->status_h + 4);
    *tc_err_h = 0;
    if (p->tc_spread) PSWF_CUDA(cudaMemcpyAsync(tc_err_h, p->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PSWF_CUDA(cudaStreamSynchronize(s));
    if (energy) *energy = p->status_h[3];
    if (*tc_err_h) return fail(EWALD_ETIMEOUT, "tensor-core spreading: an MMA completion wait ran out");
    if (p->status_h[2] > 0) return fail(EWALD_ENONFINITE, "non-finite position or charge in the input");
    if (std::fabs(p->status_h[0]) > 1e-10 * p->status_h[1])
        return fail(EWALD_ENONNEUTRAL, "charges are not neutral: |sum rho| > 1e-10 sum |rho|");
    return EWALD_OK;
}

int check_ptr_device(const void* ptr, const char* name) {
    if (!ptr) return EWALD_OK;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return fail(EWALD_EINVAL, std::string(name) + " is not a CUDA-accessible pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(EWALD_EINVAL, std::string(name) + " must be a device pointer (use ewald_eval_host for host buffers)");
    return EWALD_OK;
}

}  // namespace

namespace {

int plan_create_impl(const double* box, int64_t n, double tol, const ewald_opts* opts, ewald_plan* out,
                     const pswf::HostPlan* pre = nullptr);

// The forked streams and events of a plan's evaluation (real-space sum and Alg. 2 run concurrently).
int member_streams(ewald_plan p) {
    if (p->s_short) return EWALD_OK;
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithPriority(&p->s_short, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&p->s_alg2, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join2, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(EWALD_ECUDA, "stream/event creation failed");
    }
    return EWALD_OK;
}

// Synthetic tuning system: n uniform points in the box (xorshift64*), charges +1, -1, ... (the last
// one 0 for odd n), neutral.
void tuning_system(const double* box, int64_t n, std::vector<double>& x, std::vector<double>& rho) {
    x.resize(3 * static_cast<size_t>(n));
    rho.resize(static_cast<size_t>(n));
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (size_t i = 0; i < x.size(); ++i) {
        st ^= st >> 12;
        st ^= st << 25;
        st ^= st >> 27;
        x[i] = box[i % 3] * static_cast<double>((st * 0x2545F4914F6CDD1Dull) >> 11) * 0x1.0p-53;
    }
    for (int64_t i = 0; i < n; ++i) rho[i] = (i % 2 == 0) ? 1.0 : -1.0;
    if (n % 2) rho[n - 1] = 0.0;
}

int plan_autotune(const double* box, int64_t n, double tol, const ewald_opts& o, ewald_plan* out) {
    ewald_opts base = o;
    base.autotune = 0;
    try {
        pswf::make_plan_box(box, n, tol, base);   // argument validation before any allocation
    } catch (const std::invalid_argument& e) {
        return fail(EWALD_EINVAL, e.what());
    } catch (const std::length_error& e) {
        return fail(EWALD_ETOOBIG, e.what());
    } catch (const std::exception& e) {
        return fail(EWALD_EINVAL, e.what());
    }
    std::vector<double> xh, rh;
    tuning_system(box, n, xh, rh);
    double *xd = nullptr, *rd = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (xd) cudaFree(xd);
        if (rd) cudaFree(rd);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    };
    if (cudaMalloc(&xd, sizeof(double) * xh.size()) != cudaSuccess ||
        cudaMalloc(&rd, sizeof(double) * rh.size()) != cudaSuccess ||
        cudaMemcpy(xd, xh.data(), sizeof(double) * xh.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(rd, rh.data(), sizeof(double) * rh.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(EWALD_ENOMEM, "autotune: device allocation failed");
    }
    ewald_plan best = nullptr;
    float best_ms = 0.f;
    double best_gd = base.grid_density;
    // times one candidate (warm-up + 3 evaluations); keeps it when it is the fastest so far
    auto try_candidate = [&](const ewald_opts& c) -> int {
        ewald_plan cand = nullptr;
        if (plan_create_impl(box, n, tol, &c, &cand) != EWALD_OK) return EWALD_OK;   // not a usable shape
        int rc = eval_device(cand, xd, rd, nullptr, nullptr, st);   // warm-up
        float ms = 0.f;
        if (rc == EWALD_OK) {
            cudaEventRecord(e0, st);
            for (int k = 0; k < 3 && rc == EWALD_OK; ++k) rc = eval_device(cand, xd, rd, nullptr, nullptr, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = EWALD_ECUDA;
        }
        if (rc != EWALD_OK) {
            delete cand;
            return rc;
        }
        if (!best || ms < best_ms) {
            delete best;
            best = cand;
            best_ms = ms;
            best_gd = c.grid_density;
        } else {
            delete cand;
        }
        return EWALD_OK;
    };
    // stage 1: grid density g = m^3/n (the cutoff; Sec. 6.2.2 leaves r_c to runtime measurements)
    std::vector<int64_t> seen_m;   // grid sizes tried (m_x m_y m_z)
    for (const double gd : {1.5, 2.0, 3.0, 4.0, 6.0, 8.0, 12.0}) {
        ewald_opts c = base;
        c.grid_density = gd;
        int64_t m = 0;
        try {
            const ewald_params q = pswf::make_plan_box(box, n, tol, c).p;
            m = static_cast<int64_t>(q.grid[0]) * q.grid[1] * q.grid[2];
        } catch (const std::exception&) {
            continue;   // e.g. a grid beyond the size limit
        }
        if (std::find(seen_m.begin(), seen_m.end(), m) != seen_m.end()) continue;
        seen_m.push_back(m);
        const int rc = try_candidate(c);
        if (rc != EWALD_OK) {
            delete best;
            cleanup();
            return rc;
        }
    }
    // stage 2: the real-space cell shape (cells of edge r_c / reach) at the chosen density, unless the
    // caller fixed the reach
    if (best && base.sr_reach == 0) {
        const int r0 = best->hp.p.sr_reach;
        for (const int reach : {1, 2, 3, 4}) {
            if (reach == r0) continue;
            ewald_opts c = base;
            c.grid_density = best_gd;
            c.sr_reach = reach;
            const int rc = try_candidate(c);
            if (rc != EWALD_OK) {
                delete best;
                cleanup();
                return rc;
            }
        }
    }
    cleanup();
    if (!best) return fail(EWALD_EINVAL, "autotune: no candidate plan could be created");
    *out = best;
    return EWALD_OK;
}

// pre: the host plan computed already (batches plan their systems on several threads first)
int plan_create_impl(const double* box, int64_t n, double tol, const ewald_opts* opts, ewald_plan* out,
                     const pswf::HostPlan* pre) {
    if (!out) return fail(EWALD_EINVAL, "out is NULL");
    *out = nullptr;
    if (n > (int64_t(1) << 30)) return fail(EWALD_ETOOBIG, "n beyond 2^30 particles");
    ewald_plan p = new (std::nothrow) ewald_plan_s();
    if (!p) return fail(EWALD_ENOMEM, "host allocation failed");
    p->pooled = t_pool != nullptr;   // set before the first allocation: a failure frees nothing of the pool
    try {
        const ewald_opts o = opts ? *opts : pswf::default_opts();
        p->hp = pre ? *pre : pswf::make_plan_box(box, n, tol, o);
    } catch (const std::invalid_argument& e) {
        delete p;
        return fail(EWALD_EINVAL, e.what());
    } catch (const std::length_error& e) {
        delete p;
        return fail(EWALD_ETOOBIG, e.what());
    } catch (const std::exception& e) {
        delete p;
        return fail(EWALD_EINVAL, e.what());
    }
    // a missing device is reported as such, not as the failure of the first allocation
    int ndev = 0;
    const cudaError_t de = cudaGetDeviceCount(&ndev);
    if (de != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        delete p;
        return fail(EWALD_ECUDA, std::string("no CUDA device: ") + (de != cudaSuccess ? cudaGetErrorString(de) : "none found"));
    }
    const ewald_params& q = p->hp.p;
    p->fp64 = q.precision != EWALD_MIXED;
    p->ff = q.precision == EWALD_FLOATFLOAT;
    pswf::Geom& g = p->g;
    g.n = static_cast<int>(n);
    g.P = q.P;
    g.T = q.tile;
    g.reach = q.sr_reach;
    g.reachz = q.sr_reach_z;
    g.degw = q.deg_w;
    g.degr = q.deg_r;
    for (int d = 0; d < 3; ++d) {
        g.m[d] = q.grid[d];
        g.nt[d] = q.grid[d] / q.tile;
        g.ncell[d] = q.cells[d];
        g.L[d] = q.box[d];
        g.invL[d] = 1.0 / q.box[d];
        g.invh[d] = q.grid[d] / q.box[d];
        g.cellw[d] = q.box[d] / q.cells[d];
        g.invcellw[d] = q.cells[d] / q.box[d];
        auto split = [](double v, float (&o)[2]) {
            o[0] = static_cast<float>(v);
            o[1] = static_cast<float>(v - static_cast<double>(o[0]));
        };
        split(g.L[d], g.Lf[d]);
        split(g.invL[d], g.invLf[d]);
        split(g.invh[d], g.invhf[d]);
        split(g.cellw[d], g.cellwf[d]);
        split(g.invcellw[d], g.invcellwf[d]);
    }
    g.rc = q.rc;
    g.self = q.self_coeff;
    p->ntiles = g.nt[0] * g.nt[1] * g.nt[2];
    // x-chains of the spreading: the largest divisor of the x tile count with K T <= 32 that still leaves
    // one chain per SM (small grids take K = 1: a 3 x 3 x 3-tile grid gets 27 CTAs instead of 9); batch
    // members (pre != nullptr) keep the longest chains, since one fused launch covers all systems
    p->tc_spread = q.spread_kernel == 2;
    g.K = 1;
    const int ntiles_all = g.nt[0] * g.nt[1] * g.nt[2];
    for (int k = 32 / g.T; k >= 1; --k)
        if (g.nt[0] % k == 0 && (pre || k == 1 || ntiles_all / k >= kNumSMs)) {
            g.K = k;
            break;
        }
    p->ncells = g.ncell[0] * g.ncell[1] * g.ncell[2];
    p->m3 = static_cast<size_t>(g.m[0]) * g.m[1] * g.m[2];
    p->nspec = static_cast<size_t>(g.m[0]) * g.m[1] * (g.m[2] / 2 + 1);
    p->epart_blocks = 256;
    cudaGetDevice(&p->device);

    const size_t rs = p->fp64 ? sizeof(double) : sizeof(float);
    const int E = g.T + g.P - 1;
    const size_t m3 = p->m3, nspec = p->nspec;
    struct A { void** ptr; size_t bytes; } allocs[] = {
        {reinterpret_cast<void**>(&p->key_rank), sizeof(int4) * n},
        {reinterpret_cast<void**>(&p->perm), sizeof(int) * 2 * n},
        {&p->zeroed, sizeof(double) * 4 + sizeof(int) * (((p->ntiles + 1 + 3) / 4) * 4 + ((p->ncells + 1 + 3) / 4) * 4 + 4)},
        {reinterpret_cast<void**>(&p->tile_off), sizeof(int) * (p->ntiles + 1)},
        {reinterpret_cast<void**>(&p->cell_off), sizeof(int) * (p->ncells + 1)},
        {&p->sp_rec, 4 * rs * n},
        {reinterpret_cast<void**>(&p->sp_idx), sizeof(int2) * n},
        {&p->sr_rec, 4 * rs * n},
        {reinterpret_cast<void**>(&p->sr_idx), sizeof(int2) * n},
        {&p->scratch, rs * (static_cast<size_t>(p->ntiles) * g.T * E * E +
                            static_cast<size_t>(p->ntiles / g.K) * (E - g.T) * E * E)},
        {&p->grid_a, rs * m3},
        {&p->grid_b, rs * m3},
        {&p->spec, 2 * rs * nspec},
        {reinterpret_cast<void**>(&p->phi_int), sizeof(double) * n},
        {reinterpret_cast<void**>(&p->f_int), sizeof(double) * 3 * n},
        {reinterpret_cast<void**>(&p->epart), sizeof(double) * p->epart_blocks},
        {reinterpret_cast<void**>(&p->energy_d), sizeof(double)},
        {reinterpret_cast<void**>(&p->x_stage), sizeof(double) * 3 * n},
        {reinterpret_cast<void**>(&p->phi_sr), sizeof(double) * n},
        {reinterpret_cast<void**>(&p->f_sr), sizeof(double) * 3 * n},
        {reinterpret_cast<void**>(&p->rho_stage), sizeof(double) * n},
    };
    for (auto& a : allocs) {
        if (dmalloc(a.ptr, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            delete p;
            return fail(EWALD_ENOMEM, "device allocation failed (" + std::to_string(a.bytes) + " bytes)");
        }
    }
    // carve the zero-initialised block: status (4 doubles: sum rho, sum |rho|, non-finite count, ticket
    // counter of k_combine_energy), tile counters, cell counters (16-byte aligned)
    p->status = static_cast<double*>(p->zeroed);
    p->tile_cnt = reinterpret_cast<int*>(p->status + 4);
    p->cell_cnt = p->tile_cnt + ((p->ntiles + 1 + 3) / 4) * 4;
    p->tc_err = p->cell_cnt + ((p->ncells + 1 + 3) / 4) * 4;
    p->zeroed_bytes = sizeof(double) * 4 + sizeof(int) * (((p->ntiles + 1 + 3) / 4) * 4 + ((p->ncells + 1 + 3) / 4) * 4 + 4);
    if ((!p->fp64 && dmalloc(&p->sr_lo, 4 * sizeof(float) * n) != cudaSuccess) ||
        (p->fp64 && !p->ff && dmalloc(&p->sr_f32, sizeof(float4) * n) != cudaSuccess) ||
        (p->ff && dmalloc(&p->sr_cz, sizeof(int) * n) != cudaSuccess) ||
        (p->ff && dmalloc(&p->grid_ff, sizeof(float2) * m3) != cudaSuccess)) {
        cudaGetLastError();
        delete p;
        return fail(EWALD_ENOMEM, "device allocation failed (real-space residues)");
    }
    {
        // real-space columns: (dx, dy) within reach and, for each, the largest |dz| keeping the box
        // distance between target and source cell below rc
        std::vector<int4> cols;
        const int R = g.reach, Rz = g.reachz;
        // box distance between cells offset by (dx, dy, dz): sum_d (max(|d| - 1, 0) w_d)^2
        auto gap = [&](int k, int d) { return (k == 0 ? 0 : std::abs(k) - 1) * g.cellw[d]; };
        const double lim = g.rc * g.rc * (1.0 + 2e-4);   // a superset of what the kernels' float32 tests admit
        for (int dx = -R; dx <= R; ++dx)
            for (int dy = -R; dy <= R; ++dy) {
                const double gxy = gap(dx, 0) * gap(dx, 0) + gap(dy, 1) * gap(dy, 1);
                if (gxy >= lim) continue;
                int dzmax = 0;
                while (dzmax < Rz && gxy + gap(dzmax + 1, 2) * gap(dzmax + 1, 2) < lim) ++dzmax;
                cols.push_back(make_int4(dx, dy, dzmax, 0));
            }
        p->n_cols = static_cast<int>(cols.size());
        // every column's z-run splits into at most ceil((2R+1)/nc) + 1 contiguous pieces
        const int pieces = (2 * Rz + 1 + g.ncell[2] - 1) / g.ncell[2] + 1;
        p->sr_rcap = p->n_cols * pieces;
        if (p->sr_rcap > pswf::kShortMaxRanges) {
            delete p;
            return fail(EWALD_EINVAL, "real-space neighbourhood has too many cell ranges for the kernel");
        }
        if (dmalloc(&p->sr_cols, sizeof(int4) * cols.size()) != cudaSuccess ||
            cudaMemcpy(p->sr_cols, cols.data(), sizeof(int4) * cols.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            delete p;
            return fail(EWALD_ENOMEM, "device allocation of the real-space columns failed");
        }
    }
    if (std::max(p->ntiles, p->ncells) > kScanMulti) {   // long counter arrays: multi-block scan scratch
        p->scan_nb0 = (p->ntiles + pswf::kScanChunk - 1) / pswf::kScanChunk;
        p->scan_nb1 = (p->ncells + pswf::kScanChunk - 1) / pswf::kScanChunk;
        if (dmalloc(&p->scan_tmp, sizeof(int) * scan_tmp_ints(p->scan_nb0, p->scan_nb1)) != cudaSuccess) {
            cudaGetLastError();
            delete p;
            return fail(EWALD_ENOMEM, "device allocation of the scan scratch failed");
        }
    }
    // batch members (pre != nullptr) get their streams and events only when a batch graph is captured
    // (member_streams), and never evaluate on their own, so they need no pinned status buffer
    if (!pre) {
        const int rcs = member_streams(p);
        if (rcs != EWALD_OK) {
            delete p;
            return rcs;
        }
        if (cudaMallocHost(reinterpret_cast<void**>(&p->status_h), sizeof(double) * 5) != cudaSuccess) {
            delete p;
            return fail(EWALD_ENOMEM, "pinned host allocation failed");
        }
    }
    int rc = EWALD_OK;
    if (p->ff) {
        p->ff_kf = ff_split_index(p->hp);
        p->ff_kr = ff_radial_split(p->hp);
        if ((rc = upload_ff(reinterpret_cast<float**>(&p->wcoef), p->hp.wc)) ||
            (rc = upload_ff(reinterpret_cast<float**>(&p->dwcoef), p->hp.dwc)) ||
            (rc = upload<double>(reinterpret_cast<double**>(&p->iw), p->hp.iw)) ||
            (rc = upload<double>(reinterpret_cast<double**>(&p->mtab), p->hp.mtab)) ||
            (rc = upload<double>(reinterpret_cast<double**>(&p->gcoef), p->hp.gc))) {
            delete p;
            return rc;
        }
    } else if (p->fp64) {
        if ((rc = upload<double>(reinterpret_cast<double**>(&p->wcoef), p->hp.wc)) ||
            (rc = upload<double>(reinterpret_cast<double**>(&p->dwcoef), p->hp.dwc)) ||
            (rc = upload<double>(reinterpret_cast<double**>(&p->p1c), p->hp.p1c)) ||
            (rc = upload<double>(reinterpret_cast<double**>(&p->qc), p->hp.qc)) ||
            (rc = upload<double>(reinterpret_cast<double**>(&p->iw), p->hp.iw)) ||
            (rc = upload<double>(reinterpret_cast<double**>(&p->mtab), p->hp.mtab)) ||
            (rc = upload<double>(reinterpret_cast<double**>(&p->gcoef), p->hp.gc))) {
            delete p;
            return rc;
        }
    } else {
        if ((rc = upload<float>(reinterpret_cast<float**>(&p->wcoef), p->hp.wc)) ||
            (rc = upload<float>(reinterpret_cast<float**>(&p->dwcoef), p->hp.dwc)) ||
            (rc = upload<float>(reinterpret_cast<float**>(&p->p1c), p->hp.p1c)) ||
            (rc = upload<float>(reinterpret_cast<float**>(&p->qc), p->hp.qc)) ||
            (rc = upload<float>(reinterpret_cast<float**>(&p->iw), p->hp.iw)) ||
            (rc = upload<float>(reinterpret_cast<float**>(&p->mtab), p->hp.mtab)) ||
            (rc = upload<float>(reinterpret_cast<float**>(&p->gcoef), p->hp.gc))) {
            delete p;
            return rc;
        }
    }
    const cufftType tf = p->fp64 ? CUFFT_D2Z : CUFFT_R2C, ti = p->fp64 ? CUFFT_Z2D : CUFFT_C2R;
    size_t wf = 0, wi = 0;
    if ((rc = shared_fft(p->device, g.m, tf, &p->fwd, &wf)) || (rc = shared_fft(p->device, g.m, ti, &p->inv, &wi))) {
        delete p;
        return rc;
    }
    if (dmalloc(&p->fft_work, std::max<size_t>(std::max(wf, wi), 256)) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(EWALD_ENOMEM, "device allocation of the cuFFT work area failed");
    }
    *out = p;
    return EWALD_OK;
}

// Per-system status triple and energy of a batch, gathered for one device-to-host copy.
__global__ void k_batch_gather(const double* const* __restrict__ src, int nsys, double* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nsys) return;
    const double* st = src[2 * b];
    const double* en = src[2 * b + 1];
    out[4 * b + 0] = st[0];
    out[4 * b + 1] = st[1];
    out[4 * b + 2] = st[2];
    out[4 * b + 3] = en[0];
}

// Radial polynomials of every member, padded with leading zeros to the batch's degree bucket D.
template <int D>
std::vector<unsigned char> batch_kps(const std::vector<ewald_plan_s*>& members) {
    std::vector<unsigned char> out(sizeof(pswf::ShortParams<float, D>) * members.size());
    for (size_t i = 0; i < members.size(); ++i) {
        pswf::ShortParams<float, D> kp{};
        const ewald_plan_s* m = members[i];
        for (int k = 0; k <= D; ++k) {
            kp.p1[k] = static_cast<float>(k < static_cast<int>(m->hp.p1c.size()) ? m->hp.p1c[k] : 0.0);
            kp.q[k] = static_cast<float>(k < static_cast<int>(m->hp.qc.size()) ? m->hp.qc[k] : 0.0);
        }
        kp.rc2 = static_cast<float>(m->g.rc * m->g.rc);
        kp.two_over_rc2 = static_cast<float>(2.0 / (m->g.rc * m->g.rc));
        kp.rc2f = static_cast<float>(m->g.rc * m->g.rc * (1.0 + 1e-4));
        std::memcpy(out.data() + i * sizeof(kp), &kp, sizeof(kp));
    }
    return out;
}

// Fused evaluation (batch.cuh) for batches of float32 systems sharing the window support: descriptors,
// per-stage block tables, and for every grid size one pool of contiguous grids with batched cuFFT plans
// (the members' own grids are replaced by slices of the pool).  Batches it does not cover keep the
// captured graph of per-system pipelines.
int setup_fused(ewald_plan p) {
    const int ns = static_cast<int>(p->members.size());
    const int P = p->members[0]->g.P;
    int dmax = 0, degw = 0, rcap = 0;
    for (const ewald_plan_s* m : p->members) {
        if (m->fp64 || m->ff || m->hp.p.deg_g != 0 || m->g.P != P || m->g.T != pswf::kTile32) return EWALD_OK;
        dmax = std::max(dmax, m->g.degr);
        degw = std::max(degw, m->g.degw);
        rcap = std::max(rcap, m->sr_rcap);
    }
    const int D = dmax <= 8 ? 8 : dmax <= 10 ? 10 : dmax == 11 ? 11 : dmax <= 12 ? 12 : dmax <= 16 ? 16 : 0;
    if (D == 0 || !pswf::batch_f32_supports(P, D)) return EWALD_OK;
    // grid pools and batched cuFFT plans per grid size
    std::map<int, std::vector<int>> bym;
    for (int i = 0; i < ns; ++i) bym[p->members[i]->g.m[0]].push_back(i);
    for (const auto& kv : bym) {
        ewald_plan_s::FftGroup fg;
        fg.m = kv.first;
        fg.count = static_cast<int>(kv.second.size());
        const size_t m3 = static_cast<size_t>(fg.m) * fg.m * fg.m, nsp = static_cast<size_t>(fg.m) * fg.m * (fg.m / 2 + 1);
        if (cudaMalloc(reinterpret_cast<void**>(&fg.a), sizeof(float) * m3 * fg.count) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&fg.b), sizeof(float) * m3 * fg.count) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&fg.spec), sizeof(float2) * nsp * fg.count) != cudaSuccess) {
            cudaGetLastError();
            p->fgroups.push_back(fg);
            return fail(EWALD_ENOMEM, "fused batch: grid pool allocation failed");
        }
        int nn[3] = {fg.m, fg.m, fg.m};
        const bool ok = cufftPlanMany(&fg.fwd, 3, nn, nullptr, 1, static_cast<int>(m3), nullptr, 1,
                                      static_cast<int>(nsp), CUFFT_R2C, fg.count) == CUFFT_SUCCESS &&
                        cufftPlanMany(&fg.inv, 3, nn, nullptr, 1, static_cast<int>(nsp), nullptr, 1,
                                      static_cast<int>(m3), CUFFT_C2R, fg.count) == CUFFT_SUCCESS;
        p->fgroups.push_back(fg);
        if (!ok) return fail(EWALD_ECUFFT, "fused batch: batched cuFFT plan creation failed");
        for (int k = 0; k < fg.count; ++k) {
            ewald_plan_s* m = p->members[kv.second[k]];
            if (!m->pooled) {   // pooled members' grids stay in the batch pool (released with it)
                cudaFree(m->grid_a);
                cudaFree(m->grid_b);
                cudaFree(m->spec);
            }
            m->grid_a = fg.a + k * m3;
            m->grid_b = fg.b + k * m3;
            m->spec = fg.spec + k * nsp;
            m->pooled_grids = true;
        }
    }
    // descriptors and block tables
    std::vector<pswf::BatchSysF> sys(ns);
    std::vector<int> start(static_cast<size_t>(pswf::kBStages) * (ns + 1), 0);
    p->btotal.assign(pswf::kBStages, 0);
    const int per_short = pswf::kShortWarps * pswf::kShortTPW;
    for (int i = 0; i < ns; ++i) {
        ewald_plan_s* m = p->members[i];
        pswf::BatchSysF& b = sys[i];
        b.g = m->g;
        b.sc = scale_params<float>(m);
        b.inv_alpha = pswf::Vec4<float>{static_cast<float>(2.0 * m->g.m[0] / (P * m->g.L[0])),
                                        static_cast<float>(2.0 * m->g.m[1] / (P * m->g.L[1])),
                                        static_cast<float>(2.0 * m->g.m[2] / (P * m->g.L[2])), 0.f};
        b.key_rank = m->key_rank;
        b.perm = m->perm;
        b.tile_cnt = m->tile_cnt;
        b.tile_off = m->tile_off;
        b.cell_cnt = m->cell_cnt;
        b.cell_off = m->cell_off;
        b.status = m->status;
        b.zeroed = static_cast<int*>(m->zeroed);
        b.sp_rec = static_cast<pswf::Vec4<float>*>(m->sp_rec);
        b.sp_idx = m->sp_idx;
        b.sr_rec = static_cast<pswf::Vec4<float>*>(m->sr_rec);
        b.sr_idx = m->sr_idx;
        b.sr_lo = static_cast<pswf::Vec4<float>*>(m->sr_lo);
        b.scratch = static_cast<float*>(m->scratch);
        b.grid_a = static_cast<float*>(m->grid_a);
        b.grid_b = static_cast<float*>(m->grid_b);
        b.spec = static_cast<float2*>(m->spec);
        b.wcoef = static_cast<const float*>(m->wcoef);
        b.dwcoef = static_cast<const float*>(m->dwcoef);
        b.phi_sr = reinterpret_cast<float*>(m->phi_sr);
        b.f_sr = reinterpret_cast<float*>(m->f_sr);
        b.epart = m->epart;
        b.energy = m->energy_d;
        b.off = p->offsets[i];
        b.zeroed_ints = static_cast<int>(m->zeroed_bytes / sizeof(int));
        b.ntiles = m->ntiles;
        b.ncells = m->ncells;
        b.m3 = static_cast<int>(m->m3);
        b.nspec = static_cast<int>(m->nspec);
        b.rcap = m->sr_rcap;
        b.degw = m->g.degw;
        const int n = m->g.n, nb = (n + 255) / 256;
        b.eblocks = std::min(256, std::max(1, nb));
        const int blocks[pswf::kBStages] = {(b.zeroed_ints + 255) / 256, nb, 2, nb, 2 * nb, nb,
                                            (n + per_short - 1) / per_short, b.ntiles / m->g.K, (b.m3 + 255) / 256,
                                            (b.nspec + 255) / 256, b.ntiles, b.eblocks};
        for (int st = 0; st < pswf::kBStages; ++st) {
            start[st * (ns + 1) + i + 1] = start[st * (ns + 1) + i] + blocks[st];
        }
    }
    for (int st = 0; st < pswf::kBStages; ++st) p->btotal[st] = start[st * (ns + 1) + ns];
    // block maps: every block of every stage -> {system, local block}
    p->bmoff.assign(pswf::kBStages + 1, 0);
    for (int st = 0; st < pswf::kBStages; ++st) p->bmoff[st + 1] = p->bmoff[st] + p->btotal[st];
    std::vector<int2> bmap(static_cast<size_t>(p->bmoff[pswf::kBStages]));
    for (int st = 0; st < pswf::kBStages; ++st)
        for (int i = 0; i < ns; ++i)
            for (int k = start[st * (ns + 1) + i]; k < start[st * (ns + 1) + i + 1]; ++k)
                bmap[p->bmoff[st] + k] = make_int2(i, k - start[st * (ns + 1) + i]);
    std::vector<unsigned char> kps;
    switch (D) {
        case 8: kps = batch_kps<8>(p->members); break;
        case 10: kps = batch_kps<10>(p->members); break;
        case 11: kps = batch_kps<11>(p->members); break;
        case 12: kps = batch_kps<12>(p->members); break;
        default: kps = batch_kps<16>(p->members); break;
    }
    if (cudaMalloc(&p->bsys_d, sizeof(pswf::BatchSysF) * ns) != cudaSuccess ||
        cudaMalloc(&p->bkp_d, kps.size()) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&p->bmap_d), sizeof(int2) * std::max<size_t>(bmap.size(), 1)) != cudaSuccess ||
        cudaMemcpy(p->bsys_d, sys.data(), sizeof(pswf::BatchSysF) * ns, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->bkp_d, kps.data(), kps.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->bmap_d, bmap.data(), sizeof(int2) * bmap.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return fail(EWALD_ENOMEM, "fused batch: descriptor allocation failed");
    }
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&p->bs_short, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->bfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->bjoin, cudaEventDisableTiming) != cudaSuccess)
        return fail(EWALD_ECUDA, "fused batch: stream or event creation failed");
    p->bspread_smem = pswf::Launch<float>::spread_smem(P, degw);
    p->binterp_smem = pswf::Launch<float>::interp_smem(P, degw);
    p->bshort_smem = pswf::short_dyn_smem_f32(rcap);
    p->bD = D;
    p->bP = P;
    p->fused = true;
    return EWALD_OK;
}

int run_fused(ewald_plan p, const double* x, const double* rho, double* phi, double* f, cudaStream_t s) {
    std::vector<pswf::BatchFftF> ff;
    for (const auto& fg : p->fgroups) ff.push_back(pswf::BatchFftF{fg.count, fg.fwd, fg.inv, fg.a, fg.b, fg.spec});
    pswf::BatchRunF r{};
    r.sys = static_cast<const pswf::BatchSysF*>(p->bsys_d);
    r.kps = p->bkp_d;
    r.map = p->bmap_d;
    r.moff = p->bmoff.data();
    r.total = p->btotal.data();
    r.nsys = static_cast<int>(p->members.size());
    r.P = p->bP;
    r.D = p->bD;
    r.spread_smem = p->bspread_smem;
    r.interp_smem = p->binterp_smem;
    r.short_smem = p->bshort_smem;
    r.ffts = ff.data();
    r.nfft = static_cast<int>(ff.size());
    r.x = x;
    r.rho = rho;
    r.phi = phi;
    r.f = f;
    std::lock_guard<std::mutex> lk(fft_cache().mu);   // cuFFT handles are bound to the stream per call
    PSWF_CUDA(pswf::batch_f32_run(r, s, p->bs_short, p->bfork, p->bjoin));
    k_batch_gather<<<(r.nsys + 127) / 128, 128, 0, s>>>(p->bsrc_d, r.nsys, p->bout_d);
    PSWF_CUDA(cudaGetLastError());
    return EWALD_OK;
}

// Captures every member's pipeline into one graph: the origin stream forks to one stream per system,
// each runs eval_device (which forks further to the member's own real-space / Alg. 2 streams), and the
// origin joins them all before the gather.
int capture_batch(ewald_plan p, const double* x, const double* rho, double* phi, double* f) {
    for (ewald_plan_s* m : p->members)
        if (const int rs = member_streams(m)) return rs;
    for (size_t b = 0; b < p->bstreams.size(); ++b)
        if (!p->bstreams[b] && (cudaStreamCreateWithFlags(&p->bstreams[b], cudaStreamNonBlocking) != cudaSuccess ||
                                cudaEventCreateWithFlags(&p->bevents[b], cudaEventDisableTiming) != cudaSuccess))
            return fail(EWALD_ECUDA, "batch capture: stream or event creation failed");
    if (p->bexec) {
        cudaGraphExecDestroy(p->bexec);
        p->bexec = nullptr;
    }
    PSWF_CUDA(cudaStreamBeginCapture(p->bcap, cudaStreamCaptureModeThreadLocal));
    int rc = EWALD_OK;
    auto step = [&](cudaError_t e) {
        if (rc == EWALD_OK && e != cudaSuccess) rc = fail(EWALD_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    };
    step(cudaEventRecord(p->bstart, p->bcap));
    const int ns = static_cast<int>(p->members.size());
    for (int b = 0; b < ns && rc == EWALD_OK; ++b) {
        const size_t o = static_cast<size_t>(p->offsets[b]);
        step(cudaStreamWaitEvent(p->bstreams[b], p->bstart, 0));
        if (rc == EWALD_OK)
            rc = eval_device(p->members[b], x + 3 * o, rho + o, phi ? phi + o : nullptr, f ? f + 3 * o : nullptr,
                             p->bstreams[b]);
        step(cudaEventRecord(p->bevents[b], p->bstreams[b]));
        step(cudaStreamWaitEvent(p->bcap, p->bevents[b], 0));
    }
    if (rc == EWALD_OK) {
        k_batch_gather<<<(ns + 127) / 128, 128, 0, p->bcap>>>(p->bsrc_d, ns, p->bout_d);
        step(cudaGetLastError());
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(p->bcap, &graph);
    if (rc == EWALD_OK && ee != cudaSuccess) rc = fail(EWALD_ECUDA, std::string("batch capture: ") + cudaGetErrorString(ee));
    if (rc == EWALD_OK) {
        const cudaError_t ei = cudaGraphInstantiate(&p->bexec, graph, 0);
        if (ei != cudaSuccess) {
            p->bexec = nullptr;
            rc = fail(EWALD_ECUDA, std::string("batch graph instantiation: ") + cudaGetErrorString(ei));
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (rc == EWALD_OK) {
        p->bkey[0] = x;
        p->bkey[1] = rho;
        p->bkey[2] = phi;
        p->bkey[3] = f;
    }
    return rc;
}

}  // namespace

extern "C" {

int ewald_opts_default(ewald_opts* opts) {
    if (!opts) return fail(EWALD_EINVAL, "opts is NULL");
    *opts = pswf::default_opts();
    return EWALD_OK;
}

int ewald_plan_params_box(const double* L, int64_t n, double tol, const ewald_opts* opts, ewald_params* out) {
    if (!out || !L) return fail(EWALD_EINVAL, "NULL L or out");
    try {
        const ewald_opts o = opts ? *opts : pswf::default_opts();
        *out = pswf::make_plan_box(L, n, tol, o).p;
        return EWALD_OK;
    } catch (const std::invalid_argument& e) {
        return fail(EWALD_EINVAL, e.what());
    } catch (const std::length_error& e) {
        return fail(EWALD_ETOOBIG, e.what());
    } catch (const std::exception& e) {
        return fail(EWALD_EINVAL, e.what());
    }
}

int ewald_plan_params(double L, int64_t n, double tol, const ewald_opts* opts, ewald_params* out) {
    const double box[3] = {L, L, L};
    return ewald_plan_params_box(box, n, tol, opts, out);
}

int ewald_plan_create_box(const double* L, int64_t n, double tol, const ewald_opts* opts, ewald_plan* out) {
    if (!out) return fail(EWALD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!L) return fail(EWALD_EINVAL, "L is NULL");
    if (opts && opts->autotune == 1) return plan_autotune(L, n, tol, *opts, out);
    return plan_create_impl(L, n, tol, opts, out);
}

int ewald_plan_create(double L, int64_t n, double tol, const ewald_opts* opts, ewald_plan* out) {
    const double box[3] = {L, L, L};
    return ewald_plan_create_box(box, n, tol, opts, out);
}

int ewald_plan_query(ewald_plan plan, ewald_params* out) {
    if (!plan || !out) return fail(EWALD_EINVAL, "NULL argument");
    *out = plan->hp.p;
    return EWALD_OK;
}

int ewald_eval(ewald_plan plan, const double* x, const double* rho, double* phi, double* force, double* energy,
               void* stream) {
    if (!plan || !x || !rho) return fail(EWALD_EINVAL, "NULL plan, x or rho");
    if (plan->is_batch) return fail(EWALD_EINVAL, "batch plan: use ewald_eval_batch");
    int rc;
    if ((rc = check_ptr_device(x, "x")) || (rc = check_ptr_device(rho, "rho")) ||
        (rc = check_ptr_device(phi, "phi")) || (rc = check_ptr_device(force, "force")))
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = eval_device(plan, x, rho, phi, force, s))) return rc;
    if (energy) return read_status(plan, s, energy);
    return EWALD_OK;
}

int ewald_eval_host(ewald_plan plan, const double* x, const double* rho, double* phi, double* force, double* energy,
                    void* stream) {
    if (!plan || !x || !rho) return fail(EWALD_EINVAL, "NULL plan, x or rho");
    if (plan->is_batch) return fail(EWALD_EINVAL, "batch plan: use ewald_eval_batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = static_cast<size_t>(plan->g.n);
    PSWF_CUDA(cudaMemcpyAsync(plan->x_stage, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    PSWF_CUDA(cudaMemcpyAsync(plan->rho_stage, rho, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    int rc = eval_device(plan, plan->x_stage, plan->rho_stage, nullptr, nullptr, s);
    if (rc) return rc;
    if (phi) PSWF_CUDA(cudaMemcpyAsync(phi, plan->phi_int, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if (force) PSWF_CUDA(cudaMemcpyAsync(force, plan->f_int, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    double e = 0.0;
    rc = read_status(plan, s, &e);
    if (energy) *energy = e;
    return rc;
}

int ewald_check(ewald_plan plan, void* stream) {
    if (!plan || plan->is_batch) return fail(EWALD_EINVAL, "NULL or batch plan");
    return read_status(plan, static_cast<cudaStream_t>(stream), nullptr);
}

int ewald_debug_grid(ewald_plan plan, int which, double* host_out) {
    if (!plan || plan->is_batch || !host_out || (which != 0 && which != 1)) return fail(EWALD_EINVAL, "bad argument");
    PSWF_CUDA(cudaDeviceSynchronize());
    const size_t m3 = plan->m3;
    const void* src = which == 0 ? plan->grid_a : plan->grid_b;
    if (plan->fp64) {
        PSWF_CUDA(cudaMemcpy(host_out, src, sizeof(double) * m3, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> tmp(m3);
        PSWF_CUDA(cudaMemcpy(tmp.data(), src, sizeof(float) * m3, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < m3; ++i) host_out[i] = tmp[i];
    }
    return EWALD_OK;
}

void ewald_plan_destroy(ewald_plan plan) { delete plan; }

int ewald_plan_batch_create(int nsys, const double* L, const int64_t* n, double tol, const ewald_opts* opts,
                            ewald_plan* out) {
    if (!out) return fail(EWALD_EINVAL, "out is NULL");
    *out = nullptr;
    if (nsys < 1 || nsys > 4096) return fail(EWALD_EINVAL, "nsys must lie in [1, 4096]");
    if (!L || !n) return fail(EWALD_EINVAL, "NULL L or n");
    ewald_opts o = opts ? *opts : pswf::default_opts();
    o.autotune = 0;
    ewald_plan p = new (std::nothrow) ewald_plan_s();
    if (!p) return fail(EWALD_ENOMEM, "host allocation failed");
    p->is_batch = true;
    p->offsets.push_back(0);
    // host planning (Alg. 3, fits, tables) of the systems on parallel threads
    std::vector<pswf::HostPlan> hps(nsys);
    std::vector<std::string> errs(nsys);
    std::vector<int> codes(nsys, EWALD_OK);
    {
        const int nth = std::max(1, std::min<int>(nsys, static_cast<int>(std::thread::hardware_concurrency())));
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t)
            th.emplace_back([&, t] {
                for (int b = t; b < nsys; b += nth) {
                    try {
                        hps[b] = pswf::make_plan(L[b], n[b], tol, o);
                    } catch (const std::invalid_argument& e) {
                        codes[b] = EWALD_EINVAL;
                        errs[b] = e.what();
                    } catch (const std::length_error& e) {
                        codes[b] = EWALD_ETOOBIG;
                        errs[b] = e.what();
                    } catch (const std::exception& e) {
                        codes[b] = EWALD_EINVAL;
                        errs[b] = e.what();
                    }
                }
            });
        for (auto& t : th) t.join();
    }
    for (int b = 0; b < nsys; ++b)
        if (codes[b] != EWALD_OK) {
            delete p;
            return fail(codes[b], "system " + std::to_string(b) + ": " + errs[b]);
        }
    p->pool.reset(new (std::nothrow) DevicePool());
    if (!p->pool) {
        delete p;
        return fail(EWALD_ENOMEM, "host allocation failed");
    }
    t_pool = p->pool.get();   // the members' device buffers come from the batch's pool
    for (int b = 0; b < nsys; ++b) {
        ewald_plan m = nullptr;
        const double box[3] = {L[b], L[b], L[b]};
        const int rc = plan_create_impl(box, n[b], tol, &o, &m, &hps[b]);
        if (rc != EWALD_OK) {
            t_pool = nullptr;
            const std::string why = g_last_error;
            delete p;
            return fail(rc, "system " + std::to_string(b) + ": " + why);
        }
        m->pooled = true;
        p->members.push_back(m);
        p->offsets.push_back(p->offsets.back() + n[b]);
    }
    t_pool = nullptr;
    p->hp = p->members[0]->hp;
    p->g = p->members[0]->g;
    cudaGetDevice(&p->device);
    p->bstreams.assign(nsys, nullptr);
    p->bevents.assign(nsys, nullptr);
    // per-system capture streams are created with the graph (capture_batch), not here
    bool ok = cudaStreamCreateWithFlags(&p->bcap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&p->bstart, cudaEventDisableTiming) == cudaSuccess;
    std::vector<const double*> src(2 * static_cast<size_t>(nsys));
    for (int b = 0; b < nsys; ++b) {
        src[2 * b] = p->members[b]->status;
        src[2 * b + 1] = p->members[b]->energy_d;
    }
    ok = ok && cudaMalloc(reinterpret_cast<void**>(&p->bout_d), sizeof(double) * 4 * nsys) == cudaSuccess &&
         cudaMallocHost(reinterpret_cast<void**>(&p->bout_h), sizeof(double) * 4 * nsys) == cudaSuccess &&
         cudaMalloc(reinterpret_cast<void**>(&p->bsrc_d), sizeof(double*) * src.size()) == cudaSuccess &&
         cudaMemcpy(p->bsrc_d, src.data(), sizeof(double*) * src.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        delete p;
        return fail(EWALD_ENOMEM, "batch plan: stream, event or buffer allocation failed");
    }
    const int frc = setup_fused(p);
    if (frc != EWALD_OK) {
        delete p;
        return frc;
    }
    *out = p;
    return EWALD_OK;
}

int ewald_eval_batch(ewald_plan plan, const int64_t* offsets, const double* x, const double* rho, double* phi,
                     double* force, double* energy, void* stream) {
    if (!plan || !plan->is_batch) return fail(EWALD_EINVAL, "not a batch plan");
    if (!offsets || !x || !rho) return fail(EWALD_EINVAL, "NULL offsets, x or rho");
    const int ns = static_cast<int>(plan->members.size());
    for (int b = 0; b <= ns; ++b)
        if (offsets[b] != plan->offsets[b])
            return fail(EWALD_EINVAL, "offsets do not match the batch plan's particle counts (entry " +
                                          std::to_string(b) + ")");
    int rc;
    if ((rc = check_ptr_device(x, "x")) || (rc = check_ptr_device(rho, "rho")) ||
        (rc = check_ptr_device(phi, "phi")) || (rc = check_ptr_device(force, "force")))
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->fused && phi && force) {
        if ((rc = run_fused(plan, x, rho, phi, force, s))) return rc;
    } else {
        if (!plan->bexec || plan->bkey[0] != x || plan->bkey[1] != rho || plan->bkey[2] != phi || plan->bkey[3] != force)
            if ((rc = capture_batch(plan, x, rho, phi, force))) return rc;
        PSWF_CUDA(cudaGraphLaunch(plan->bexec, s));
    }
    PSWF_CUDA(cudaMemcpyAsync(plan->bout_h, plan->bout_d, sizeof(double) * 4 * ns, cudaMemcpyDeviceToHost, s));
    PSWF_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < ns; ++b) {
        const double* o = plan->bout_h + 4 * b;
        if (energy) energy[b] = o[3];
        if (o[2] > 0) return fail(EWALD_ENONFINITE, "system " + std::to_string(b) + ": non-finite position or charge");
        if (std::fabs(o[0]) > 1e-10 * o[1])
            return fail(EWALD_ENONNEUTRAL, "system " + std::to_string(b) + ": charges are not neutral");
    }
    return EWALD_OK;
}

int ewald_profile(ewald_plan plan, int enable) {
    if (!plan || plan->is_batch) return fail(EWALD_EINVAL, "NULL or batch plan");
    if (enable) {
        PSWF_CUDA(cudaDeviceSynchronize());
        plan->clear_prof();
    }
    if (enable < 0 || enable > 2) return fail(EWALD_EINVAL, "enable must be 0, 1 or 2");
    plan->profiling = enable != 0;
    plan->serial = enable == 2;
    return EWALD_OK;
}

int ewald_profile_read(ewald_plan plan, double* ms, int* count) {
    if (!plan || !ms) return fail(EWALD_EINVAL, "bad argument");
    for (int k = 0; k < EWALD_NSTAGES; ++k) ms[k] = 0.0;
    for (auto& v : plan->prof) {
        for (int k = 0; k < EWALD_NSTAGES; ++k) {
            PSWF_CUDA(cudaEventSynchronize(v[2 * k + 1]));
            float t = 0.f;
            PSWF_CUDA(cudaEventElapsedTime(&t, v[2 * k], v[2 * k + 1]));
            ms[k] += t;
        }
    }
    if (count) *count = static_cast<int>(plan->prof.size());
    return EWALD_OK;
}

int ewald_debug_wait_timeout(void) {
    int* flag = nullptr;
    int h = 0;
    if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return fail(EWALD_ENOMEM, "device allocation failed");
    cudaError_t e = pswf::launch_wait_probe(20000000ll, flag, nullptr);   // ~10 ms of SM clocks
    if (e == cudaSuccess) e = cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(flag);
    if (e != cudaSuccess) return fail(EWALD_ECUDA, cudaGetErrorString(e));
    return h ? fail(EWALD_ETIMEOUT, "bounded device wait ran out (as intended: nothing arrives on the barrier)")
             : EWALD_OK;
}

// The host-table entry points take an ewald_params from the caller: everything the planner never
// produces is rejected before a table is built (a negative degree or window support would size or index
// the fitted tables out of range).
static int check_table_params(const ewald_params* p) {
    if (!p) return fail(EWALD_EINVAL, "NULL parameters");
    if (p->P < pswf::kPMin || p->P > pswf::kPMax)
        return fail(EWALD_EINVAL, "window support P must lie in [" + std::to_string(pswf::kPMin) + ", " +
                                      std::to_string(pswf::kPMax) + "]");
    if (p->deg_w < 1 || p->deg_w > pswf::kDegWMax || p->deg_r < 1 || p->deg_r > pswf::kDegRMax ||
        p->deg_g < 0 || p->deg_g > pswf::kDegRMax)
        return fail(EWALD_EINVAL, "polynomial degree outside the planner's range");
    if (!(p->cs > 0) || !(p->cw > 0) || !(p->rc > 0) || !(p->L > 0) || !(p->h > 0) || !(p->alpha > 0) ||
        !std::isfinite(p->cs) || !std::isfinite(p->cw) || !std::isfinite(p->rc) || !std::isfinite(p->L))
        return fail(EWALD_EINVAL, "bandlimits, cutoff, box edge, spacing and window half-width must be positive");
    for (int d = 0; d < 3; ++d)
        if (p->grid[d] < 4 || p->grid[d] > 1024 || !(p->box[d] > 0) || !std::isfinite(p->box[d]))
            return fail(EWALD_EINVAL, "grid sizes must lie in [4, 1024] and box edges be positive");
    if (p->m != p->grid[0] || p->L != p->box[0])
        return fail(EWALD_EINVAL, "m and L must be the x-axis entries of grid and box");
    return EWALD_OK;
}

int ewald_pswf_eval(double c, int nx, const double* x, double* psi, double* dpsi, double* chi, double* lambda0) {
    if (nx < 0 || (nx > 0 && !x)) return fail(EWALD_EINVAL, "bad point array");
    try {
        const pswf::Prolate f(c);
        for (int i = 0; i < nx; ++i) {
            if (psi) psi[i] = f.psi(x[i]);
            if (dpsi) dpsi[i] = f.dpsi(x[i]);
        }
        if (chi) *chi = f.chi;
        if (lambda0) *lambda0 = f.lambda;
        return EWALD_OK;
    } catch (const std::exception& e) {
        return fail(EWALD_EINVAL, e.what());
    }
}

double ewald_lambertw(int branch, double z) {
    try {
        return pswf::lambert_w(branch, z);
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return std::nan("");
    }
}

int ewald_window_fit(const ewald_params* p, int nz, const double* z, double* w, double* dw) {
    if (!p || nz < 0 || (nz > 0 && (!z || !w))) return fail(EWALD_EINVAL, "bad argument");
    if (const int rc = check_table_params(p)) return rc;
    try {
        const pswf::Prolate pw(p->cw);
        const auto wc = pswf::fit_window(pw, p->P, p->deg_w, false, nullptr);
        const auto dwc = pswf::fit_window(pw, p->P, p->deg_w, true, nullptr);
        const int d = p->deg_w;
        for (int i = 0; i < nz; ++i)
            for (int a = 0; a < p->P; ++a) {
                w[static_cast<size_t>(i) * p->P + a] = pswf::horner(wc.data() + a * (d + 1), d, z[i]);
                if (dw) dw[static_cast<size_t>(i) * p->P + a] = pswf::horner(dwc.data() + a * (d + 1), d, z[i]) / p->alpha;
            }
        return EWALD_OK;
    } catch (const std::exception& e) {
        return fail(EWALD_EINVAL, e.what());
    }
}

int ewald_radial_fit(const ewald_params* p, int nr, const double* r, double* R, double* G) {
    if (!p || nr < 0 || (nr > 0 && (!r || !R))) return fail(EWALD_EINVAL, "bad argument");
    if (const int rc = check_table_params(p)) return rc;
    try {
        const pswf::Prolate ps(p->cs);
        const auto c1 = pswf::fit_radial(ps, p->rc, p->deg_r, 0, nullptr);
        const auto c2 = pswf::fit_radial(ps, p->rc, p->deg_r, 1, nullptr);
        for (int i = 0; i < nr; ++i) {
            const double u = 2.0 * r[i] * r[i] / (p->rc * p->rc) - 1.0;
            R[i] = 1.0 / r[i] - pswf::horner(c1.data(), p->deg_r, u);
            if (G) G[i] = 1.0 / (r[i] * r[i] * r[i]) + pswf::horner(c2.data(), p->deg_r, u);
        }
        return EWALD_OK;
    } catch (const std::exception& e) {
        return fail(EWALD_EINVAL, e.what());
    }
}

int ewald_scale_table(const ewald_params* p, double* S) {
    if (!p || !S) return fail(EWALD_EINVAL, "bad argument");
    if (const int rc = check_table_params(p)) return rc;
    try {
        const pswf::Prolate ps(p->cs), pw(p->cw);
        std::vector<double> iw, mtab;
        pswf::scale_tables(*p, ps, pw, iw, mtab);
        if (p->deg_g > 0) {
            // cuboid: the scaling step's formula (k_scale) on the host, every mode inside the
            // mollifier's band |omega| < c_s / r_c, M-hat from the plan's polynomial of gammahat
            const std::vector<double> gc = pswf::fit_gamma(ps, p->deg_g, nullptr);
            const int mx = p->grid[0], my = p->grid[1], mz = p->grid[2], mh = mz / 2 + 1;
            const double pi = 3.14159265358979323846;
            const double V = p->box[0] * p->box[1] * p->box[2], ts = (p->rc / p->cs) * (p->rc / p->cs);
            double w2d[3];
            for (int d = 0; d < 3; ++d) w2d[d] = (2.0 * pi / p->box[d]) * (2.0 * pi / p->box[d]);
            for (int ix = 0; ix < mx; ++ix)
                for (int iy = 0; iy < my; ++iy)
                    for (int iz = 0; iz < mh; ++iz) {
                        const int kx = ix < mx / 2 ? ix : ix - mx, ky = iy < my / 2 ? iy : iy - my, kz = iz;
                        const double w2 = w2d[0] * kx * kx + w2d[1] * ky * ky + w2d[2] * kz * kz, t = w2 * ts;
                        double s = 0.0;
                        if (w2 > 0.0 && t < 1.0) {
                            const double u = 2.0 * t - 1.0;
                            double gh = gc[p->deg_g];
                            for (int k = p->deg_g - 1; k >= 0; --k) gh = gh * u + gc[k];
                            s = 4.0 * pi / V / w2 * gh * iw[ix] * iw[mx + iy] * iw[mx + my + iz];
                        }
                        S[(static_cast<size_t>(ix) * my + iy) * mh + iz] = s;
                    }
            return EWALD_OK;
        }
        const int m = p->m, mh = m / 2 + 1, qmax = (m / 2) * (m / 2);
        for (int ix = 0; ix < m; ++ix)
            for (int iy = 0; iy < m; ++iy)
                for (int iz = 0; iz < mh; ++iz) {
                    const int kx = ix < m / 2 ? ix : ix - m, ky = iy < m / 2 ? iy : iy - m, kz = iz;
                    const int q = kx * kx + ky * ky + kz * kz;
                    S[(static_cast<size_t>(ix) * m + iy) * mh + iz] =
                        (q > 0 && q < qmax) ? mtab[q] * iw[ix] * iw[iy] * iw[iz] : 0.0;
                }
        return EWALD_OK;
    } catch (const std::exception& e) {
        return fail(EWALD_EINVAL, e.what());
    }
}

const char* ewald_error_string(int code) {
    switch (code) {
        case EWALD_OK: return "ok";
        case EWALD_EINVAL: return "invalid argument";
        case EWALD_ENONNEUTRAL: return "charges are not neutral";
        case EWALD_ENOMEM: return "out of memory";
        case EWALD_ECUDA: return "CUDA runtime error";
        case EWALD_ECUFFT: return "cuFFT error";
        case EWALD_ETOOBIG: return "problem beyond library limits";
        case EWALD_ETIMEOUT: return "device wait timed out";
        case EWALD_ENONFINITE: return "non-finite input";
        default: return "unknown error";
    }
}

const char* ewald_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
