// Allocation-free spreading entry point (ewald_spread_static).
//
// Some callers cannot allocate device memory at the moment they need a result: code running
// under a custom or pre-reserved device allocator that forbids cudaMalloc/cudaFree on the hot
// path, plugins loaded into a host application that owns all GPU memory, and real-time loops
// that must not trigger the implicit synchronisation cudaMalloc/cudaFree can cause.  For them
// this entry point spreads charges onto a caller-owned grid using only a fixed scratch area
// that lives in this library's image: one file-scope __device__ array, created when a GPU first
// loads the library and held until the process exits.
//
// The computation is the float64 spreading of the regular pipeline (counting sort into tiles,
// the tile spreading kernel, the halo sum), with every intermediate buffer carved out of the
// static array instead of a plan workspace.
#include <cuda_runtime.h>

#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "device.cuh"
#include "launch.h"
#include "planner.h"
#include "pswf_ewald.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch, looked up once per device.  In host code the symbol
// name only stands in for the array; kernels must be given this address instead.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};

// The window table sits at the start of the array (offset 0, sized for the largest P and degree) and
// stays there between calls: a call whose (c_w, P, deg_w) equal the table already in place on this
// device neither refits the window on the host nor copies it.
struct TableKey {
    bool valid = false;
    double cw = 0.0;
    int P = 0, deg_w = 0;
};
TableKey g_table[kMaxDevices];

int fail_static(int code, const std::string& msg) {
    pswf::record_error(msg);   // reported by ewald_last_error()
    return code;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" int ewald_spread_static(const ewald_params* p, const double* x, const double* rho, double* grid,
                                   void* stream) {
    if (!p || !x || !rho || !grid) return fail_static(EWALD_EINVAL, "NULL argument");
    if (p->n < 1 || p->n > (int64_t(1) << 30)) return fail_static(EWALD_EINVAL, "particle count out of range");
    if (p->tile == pswf::kTile32)
        return fail_static(EWALD_EINVAL, "parameters of a float32 (EWALD_MIXED, tile 8) plan: ewald_spread_static "
                                         "takes the parameters of EWALD_FP64 or EWALD_FLOATFLOAT plans (tile 4)");
    if (p->P < pswf::kPMin || p->P > pswf::kPMax || p->tile != pswf::kTile64 || p->m % p->tile != 0 ||
        p->deg_w < 1 || p->deg_w > pswf::kDegWMax || !(p->L > 0) || !(p->alpha > 0))
        return fail_static(EWALD_EINVAL, "parameters do not come from ewald_plan_params");
    if (!(p->box[0] == p->L && p->box[1] == p->L && p->box[2] == p->L && p->grid[0] == p->m && p->grid[1] == p->m &&
          p->grid[2] == p->m))
        return fail_static(EWALD_EINVAL, "ewald_spread_static takes cubic boxes only");

    // ---- carve the static array: counts, offsets, sort records, tile slabs, window table
    const int64_t n = p->n;
    const int m = p->m, P = p->P, T = p->tile, nt = m / T, E = T + P - 1;
    const size_t ntiles = size_t(nt) * nt * nt;
    const size_t need_coef = align256(sizeof(double) * pswf::kPMax * (pswf::kDegWMax + 1));   // fixed slot
    const size_t need_key = align256(sizeof(int4) * n);
    const size_t need_perm = align256(sizeof(int) * 2 * n);
    const size_t need_tcnt = align256(sizeof(int) * (ntiles + 1));
    const size_t need_ccnt = align256(sizeof(int) * 2);
    const size_t need_status = align256(sizeof(double) * 4);
    const size_t need_rec = align256(sizeof(pswf::Vec4<double>) * n);
    const size_t need_idx = align256(sizeof(int2) * n);
    // x-chains of the spreading, as in the single-system plans: the largest divisor of nt with K T <= 32
    // that leaves one chain per SM (152), K = 1 otherwise
    int K = 1;
    for (int k = 32 / T; k >= 1; --k)
        if (nt % k == 0 && (k == 1 || ntiles / k >= 152)) {
            K = k;
            break;
        }
    const size_t need_slab = align256(sizeof(double) * (ntiles * size_t(T) * E * E +
                                                        (ntiles / K) * size_t(E - T) * E * E));
    const size_t need = need_coef + need_key + need_perm + 2 * need_tcnt + 2 * need_ccnt + need_status +
                        2 * need_rec + 2 * need_idx + need_slab;
    if (need > kStaticScratchBytes)
        return fail_static(EWALD_ETOOBIG, "ewald_spread_static needs " + std::to_string(need) +
                                              " bytes of scratch; its static array holds " +
                                              std::to_string(kStaticScratchBytes) + " bytes");

    // ---- per-device set-up: look up the array's device address with that device current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail_static(EWALD_ECUDA, "no usable current CUDA device");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev]) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess || !ptr)
                return fail_static(EWALD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = ptr;
        }
        base = g_addr[dev];
    }

    unsigned char* cur = static_cast<unsigned char*>(base);
    auto take = [&](size_t b) {
        unsigned char* r = cur;
        cur += b;
        return r;
    };
    double* coef = reinterpret_cast<double*>(take(need_coef));
    int* key_rank = reinterpret_cast<int*>(take(need_key));
    int* perm = reinterpret_cast<int*>(take(need_perm));
    int* tile_cnt = reinterpret_cast<int*>(take(need_tcnt));
    int* tile_off = reinterpret_cast<int*>(take(need_tcnt));
    int* cell_cnt = reinterpret_cast<int*>(take(need_ccnt));
    int* cell_off = reinterpret_cast<int*>(take(need_ccnt));
    double* status = reinterpret_cast<double*>(take(need_status));
    auto* sp_rec = reinterpret_cast<pswf::Vec4<double>*>(take(need_rec));
    auto* sr_rec = reinterpret_cast<pswf::Vec4<double>*>(take(need_rec));
    int2* sp_idx = reinterpret_cast<int2*>(take(need_idx));
    int2* sr_idx = reinterpret_cast<int2*>(take(need_idx));
    double* slab = reinterpret_cast<double*>(take(need_slab));

    // ---- window polynomial table (host fit, copied into the static array unless already there)
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        TableKey& tk = g_table[dev];
        if (!(tk.valid && tk.cw == p->cw && tk.P == P && tk.deg_w == p->deg_w)) {
            std::vector<double> wc;
            try {
                const pswf::Prolate pw(p->cw);
                wc = pswf::fit_window(pw, P, p->deg_w, false, nullptr);
            } catch (const std::exception& e) {
                return fail_static(EWALD_EINVAL, e.what());
            }
            tk.valid = false;
            if (cudaMemcpyAsync(coef, wc.data(), sizeof(double) * wc.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
                return fail_static(EWALD_ECUDA, "window table copy failed");
            tk = TableKey{true, p->cw, P, p->deg_w};
        }
    }

    // the array keeps the previous call's contents: counters must start at zero
    if (cudaMemsetAsync(tile_cnt, 0, sizeof(int) * ntiles, s) != cudaSuccess ||
        cudaMemsetAsync(cell_cnt, 0, sizeof(int) * 2, s) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(double) * 4, s) != cudaSuccess)
        return fail_static(EWALD_ECUDA, "clearing the static counters failed");

    pswf::Geom g{};
    g.n = static_cast<int>(n);
    g.P = P;
    g.T = T;
    g.reach = 1;
    g.reachz = 1;
    g.K = K;
    g.degw = p->deg_w;
    g.degr = 0;
    for (int d = 0; d < 3; ++d) {
        g.m[d] = m;
        g.nt[d] = nt;
        g.ncell[d] = 1;
        g.L[d] = p->L;
        g.invL[d] = 1.0 / p->L;
        g.invh[d] = m / p->L;
        g.cellw[d] = p->L;
        g.invcellw[d] = 1.0 / p->L;
    }
    g.rc = p->rc;
    g.self = 0.0;

    const int tb = 256, nb = static_cast<int>((n + tb - 1) / tb);
    pswf::k_prep<false><<<nb, tb, 0, s>>>(x, rho, g, key_rank, tile_cnt, cell_cnt, status);
    pswf::k_scan<<<2, 1024, 0, s>>>(tile_cnt, tile_off, static_cast<int>(ntiles), cell_cnt, cell_off, 1);
    // input order inside every tile (the regular pipeline's stable ranks; the single real-space cell of
    // this entry point is never read, so its ranks stay as placed)
    pswf::k_place<<<nb, tb, 0, s>>>(key_rank, static_cast<int>(n), tile_off, cell_off, perm);
    pswf::k_rerank<<<dim3(nb, 1), tb, 0, s>>>(key_rank, static_cast<int>(n), tile_off, cell_off, perm);
    pswf::k_scatter<double><<<nb, tb, 0, s>>>(x, rho, g, key_rank, tile_off, cell_off, sp_rec, sp_idx, sr_rec,
                                              sr_idx, nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_static(EWALD_ECUDA, std::string("sort launch: ") + cudaGetErrorString(e));
    e = pswf::Launch<double>::spread(P, static_cast<int>(ntiles), sp_rec, sp_idx, tile_off, coef, p->deg_w,
                                     pswf::SpreadChain{K, nt * nt, static_cast<int>(ntiles)}, slab, s);
    if (e != cudaSuccess) return fail_static(EWALD_ECUDA, std::string("spread launch: ") + cudaGetErrorString(e));
    const int mm = m * m * m;
    pswf::k_halo<double, 0><<<(mm + 255) / 256, 256, 0, s>>>(slab, tile_off, g, grid);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_static(EWALD_ECUDA, std::string("halo launch: ") + cudaGetErrorString(e));
    return EWALD_OK;
}
