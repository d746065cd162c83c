// tpc_links_noalloc: the Cellular-Automaton link finding of one event (grid
// build, neighbour finder, cleaner) with every intermediate buffer in a
// fixed, file-scope device array instead of memory allocated per call.
//
// Some callers cannot allocate device memory while they run: components of
// an online trigger or readout chain whose device memory is divided among
// components once at start-up, and latency-critical loops where cudaMalloc
// or cudaFree would synchronize the device and add unbounded delays.  This
// entry point serves them: it calls no cudaMalloc, cudaFree or other
// allocating routine; the caller passes device inputs and outputs.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "tpc_dev.cuh"

using namespace tpc;

namespace {

constexpr int kNoallocMaxClusters = TPC_NOALLOC_MAX_CLUSTERS;
constexpr size_t kScratchBytes = TPC_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxRows = 16384;  // n_sectors * n_rows of one event

// The scratch: one copy per device that loads this library's device code,
// held until the process exits.  Host code must not use this name as an
// address; it takes the device address from cudaGetSymbolAddress (see
// scratch_address).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;                       // one call at a time, see the header
int g_plan[2 * (kNoallocMaxRows + 1)]; // host plan (row and bin-table offsets)
int g_counters[kNumCounters];

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Device address of the scratch on the current device, looked up on every
// call (a table lookup once the module is loaded; a stored address would
// dangle after the device's context is torn down and recreated).  CUDA
// loads device code lazily: the first lookup on a device loads this
// library's module there, and with it the scratch array, which can fail for
// lack of device memory.
int scratch_address(void** out)
{
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TPC_ERR_NOMEM : TPC_ERR_DEVICE;
    }
    *out = ptr;
    return TPC_OK;
}

bool params_ok(const tpc_params& P)
{
    const int t = P.threads_per_row;
    return P.k_win > 0 && P.d_max2 >= 0 && P.l_seed >= 2 && P.y_margin >= 0 &&
           P.bin_target > 0 && P.bin_target < 1e6f && (t == 32 || t == 64 || t == 128 || t == 256);
}

}  // namespace

extern "C" int tpc_links_noalloc(const tpc_geometry* g, const tpc_params* params,
                                 const tpc_cluster* d_clusters, const int32_t* row_counts,
                                 int32_t* d_links, void* cuda_stream)
{
    if (!g || !row_counts || !g->row_x) return TPC_ERR_INVALID;
    const int NR = g->n_rows, S = g->n_sectors;
    if (NR < 3 || NR > TPC_MAX_ROWS || S < 2 || (S & 1) || (int64_t)S * NR > kNoallocMaxRows)
        return TPC_ERR_INVALID;
    if (!(g->tan_half_open > 0) || !(g->z_max > 0)) return TPC_ERR_INVALID;
    tpc_params P;
    tpc_params_default(&P);
    if (params) P = *params;
    if (!params_ok(P)) return TPC_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(d_clusters) & 15) return TPC_ERR_INVALID;

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // every call synchronizes with its own work, which a capturing stream
    // does not allow: refuse before enqueuing anything
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return TPC_ERR_INVALID;
    }

    std::lock_guard<std::mutex> lock(g_mu);
    // plan on the host: row CSR offsets and bin-table offsets
    const int R = S * NR;
    int* plan_off = g_plan;
    int* plan_bins = g_plan + R + 1;
    int64_t N = 0, bins = 0;
    int max_row = 1, max3 = 1, max_slots = 4, max_slots_nb = 12;
    for (int r = 0; r < R; r++) {
        const int c = row_counts[r];
        if (c < 0 || c > TPC_MAX_ROW_CLUSTERS) return TPC_ERR_INVALID;
        plan_off[r] = (int)N;
        plan_bins[r] = (int)bins;
        N += c;
        const int slots = row_bin_slots(c, P.bin_target);
        bins += slots;
        if (c > max_row) max_row = c;
        if (slots > max_slots) max_slots = slots;
        const int rr = r % NR;
        if (rr >= 1 && rr + 1 < NR) {
            const int c3 = row_counts[r - 1] + c + row_counts[r + 1];
            if (c3 > max3) max3 = c3;
            const int s2 = row_bin_slots(row_counts[r - 1], P.bin_target) +
                           row_bin_slots(row_counts[r + 1], P.bin_target);
            if (s2 > max_slots_nb) max_slots_nb = s2;
        }
    }
    if (N > kNoallocMaxClusters) return TPC_ERR_INVALID;  // beyond the fixed scratch
    plan_off[R] = (int)N;
    plan_bins[R] = (int)bins;
    // the scratch on this device, also for an empty event: an empty call at
    // start-up loads it
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TPC_ERR_DEVICE;
    void* base_v = nullptr;
    int rc = scratch_address(&base_v);
    if (rc != TPC_OK) return rc;
    char* base = static_cast<char*>(base_v);
    if (N == 0) {
        // the kernels too: an empty call leaves nothing to load later
        cudaError_t e = tpc_int::preload_link_kernels();
        if (e == cudaSuccess) e = P.exact_fp32 ? tpc_exact::preload_neighbours() : tpc_fast::preload_neighbours();
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? TPC_ERR_NOMEM : TPC_ERR_DEVICE;
        }
        return TPC_OK;
    }
    if (!d_clusters || !d_links) return TPC_ERR_INVALID;

    // lay out the scratch
    const size_t n = (size_t)N;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align256(off + (bytes < 16 ? 16 : bytes));
        return at;
    };
    const size_t o_rowx = take(sizeof(float) * TPC_MAX_ROWS);
    const size_t o_cnt = take((size_t)R * 4);
    const size_t o_plan = take((size_t)(R + 1) * 8);
    const size_t o_grid = take((size_t)R * sizeof(RowGrid));
    const size_t o_hits = take(n * 16);
    const size_t o_hyz = take((n + 2) * 8);  // + a pad entry read by whole-pair copies
    const size_t o_bins = take((size_t)bins * 4);
    const size_t o_up = take(n * 4), o_dn = take(n * 4), o_up2 = take(n * 4), o_dn2 = take(n * 4);
    const size_t o_start = take(n * 4);
    const size_t o_nstart = take((size_t)R * 4);
    const size_t o_owner = take(n * 4);
    const size_t o_count = take(kNumCounters * 4);
    if (off > kScratchBytes) return TPC_ERR_NOMEM;  // bin tables too large at this bin_target

    KConst k;
    std::memset(&k, 0, sizeof k);
    k.k_win = P.k_win;
    k.d_max2 = P.d_max2;
    k.y_margin = P.y_margin;
    k.tan_h = g->tan_half_open;
    k.z_max = g->z_max;
    k.bin_target = P.bin_target;
    k.l_seed = P.l_seed;
    k.n_rows = NR;
    k.n_sectors = S;

    DevPtrs p;
    std::memset(&p, 0, sizeof p);
    p.clusters = reinterpret_cast<const float4*>(d_clusters);
    p.row_cnt = reinterpret_cast<const int*>(base + o_cnt);
    p.row_off = reinterpret_cast<const int*>(base + o_plan);
    p.bin_cap_off = p.row_off + (R + 1);
    p.grid = reinterpret_cast<RowGrid*>(base + o_grid);
    p.hits = reinterpret_cast<float4*>(base + o_hits);
    p.hyz = reinterpret_cast<float2*>(base + o_hyz);
    p.bin_off = reinterpret_cast<int*>(base + o_bins);
    p.up = reinterpret_cast<int*>(base + o_up);
    p.dn = reinterpret_cast<int*>(base + o_dn);
    p.up2 = reinterpret_cast<int*>(base + o_up2);
    p.dn2 = reinterpret_cast<int*>(base + o_dn2);
    p.start_list = reinterpret_cast<int*>(base + o_start);
    p.row_nstart = reinterpret_cast<int*>(base + o_nstart);
    p.owner = reinterpret_cast<unsigned*>(base + o_owner);
    p.counters = reinterpret_cast<int*>(base + o_count);
    p.N = (int)N;
    p.R = R;
    p.n_units = S;

    const float* xd = reinterpret_cast<const float*>(base + o_rowx);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // Every call starts from these uploads; what must start at zero (the
    // counters) is cleared by the plan kernel, and every other scratch entry
    // a later kernel reads is written earlier in the same call.
    cudaError_t e = cudaMemcpyAsync(base + o_rowx, g->row_x, sizeof(float) * NR, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_cnt, row_counts, (size_t)R * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_plan, g_plan, (size_t)(R + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = tpc_int::launch_plan(k, xd, p, nsm, s);
    if (e == cudaSuccess) e = tpc_int::launch_grid(k, xd, p, max_row, max_slots, P.threads_per_row, 0, S, s);
    if (e == cudaSuccess)
        e = P.exact_fp32 ? tpc_exact::launch_neighbours(k, xd, p, max3, max_slots_nb, P.threads_per_row, 1, 0, S, s)
                         : tpc_fast::launch_neighbours(k, xd, p, max3, max_slots_nb, P.threads_per_row, 1, 0, S, s);
    if (e == cudaSuccess) e = tpc_int::launch_clean(k, p, P.threads_per_row, 0, S, true, s);
    if (e == cudaSuccess) e = tpc_int::launch_dump_links(p, 1, d_links, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g_counters, p.counters, sizeof g_counters, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TPC_ERR_DEVICE;
    }
    if (g_counters[C_ERR] & E_INPUT) return TPC_ERR_INVALID;
    if (g_counters[C_ERR] & E_TIMEOUT) return TPC_ERR_TIMEOUT;
    return TPC_OK;
}
