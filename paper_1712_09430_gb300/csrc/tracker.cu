// Host side of the C ABI (include/tpc_tracker.h): tracker lifecycle, device
// workspace, the batched and the plain per-sector launch sequences, CUDA-graph
// replay, output fetch with the estimate-then-fetch-the-rest scheme of
// Sec. 3.1, per-stage dumps and stage timing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tpc_dev.cuh"
#include "tpc_serve.h"

using namespace tpc;

static std::mutex g_err_mu;
static std::string g_create_err;

#define TPC_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, std::string(#call ": ") +      \
                                                                  cudaGetErrorString(e_));    \
    } while (0)

namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

// ---------------------------------------------------------------- tracker

int tpc_tracker::fail(int code, const std::string& msg)
{
    err = msg;
    return code;
}

static KConst make_kconst(const tpc_params& P, const tpc_geometry& G, double bz)
{
    KConst k;
    k.k_win = P.k_win;
    k.d_max2 = P.d_max2;
    k.sy2 = P.sigma_y * P.sigma_y;
    k.sz2 = P.sigma_z * P.sigma_z;
    k.var_s = P.var_s;
    k.var_q = P.var_q;
    k.var_t = P.var_t;
    k.n_sigma = P.n_sigma;
    k.w_min = P.w_min;
    k.w_max = P.w_max;
    k.s_max = P.s_max;
    k.y_margin = P.y_margin;
    k.kB = (float)(-0.00299792458 * bz);
    k.kP = (float)(-0.00299792458);
    for (int i = 0; i < 5; i++) k.fb[i] = P.field[i];
    k.mg_chi2 = P.merge_chi2;
    k.mg_gap = P.merge_gap;
    k.mg_overlap = P.merge_overlap;
    k.mg_window = P.merge_window;
    k.mg_on = P.merge;
    k.t0_ycut = P.t0_y_cut;
    k.t0_bin = P.t0_bin;
    k.t0_radius = P.t0_radius;
    k.t0_window = P.t0_window;
    k.t0_nmin = P.t0_n_min;
    k.t0_nb = P.t0_bin > 0 ? (int)std::ceil(2.0 * (double)G.z_max / (double)P.t0_bin) : 1;
    // angle between adjacent sectors of one side: 360 deg / (n_sectors / 2)
    const double deg = 720.0 / (double)G.n_sectors;
    const double th = deg * (3.14159265358979323846 / 180.0);
    k.mg_cos = (float)std::cos(th);
    k.mg_sin = (float)std::sin(th);
    k.tan_h = G.tan_half_open;
    k.z_max = G.z_max;
    k.bin_target = P.bin_target;
    k.l_seed = P.l_seed;
    k.g_max = P.g_max;
    k.n_min_tracklet = P.n_min_tracklet;
    k.n_min_track = P.n_min_track;
    k.own_num = P.own_num;
    k.own_den = P.own_den;
    k.n_rows = G.n_rows;
    k.n_sectors = G.n_sectors;
    k.wait_polls = (unsigned)P.debug_wait_polls;
    return k;
}

static const char* check_params(const tpc_params& P)
{
    if (!(P.k_win > 0 && P.d_max2 >= 0 && P.sigma_y > 0 && P.sigma_z > 0)) return "k_win, d_max2, sigma";
    if (!(P.var_s > 0 && P.var_q > 0 && P.var_t > 0)) return "initial variances must be > 0";
    if (!(P.n_sigma > 0 && P.w_min > 0 && P.w_max >= P.w_min)) return "search window";
    if (!(P.s_max > 0 && P.s_max < 1)) return "s_max must be in (0, 1)";
    if (!(P.y_margin >= 0)) return "y_margin";
    if (P.l_seed < 2 || P.g_max < 0 || P.n_min_tracklet < 1 || P.n_min_track < 1) return "counts";
    if (P.own_num < 0 || P.own_den < 1) return "own_num/own_den";
    if (!(P.bin_target > 0 && P.bin_target < 1e6f)) return "bin_target";
    int t = P.threads_per_row;
    if (t != 32 && t != 64 && t != 128 && t != 256) return "threads_per_row must be 32, 64, 128 or 256";
    int w = P.tracklets_per_warp;
    if (w != 1 && w != 2 && w != 4 && w != 8 && w != 16 && w != 32) return "tracklets_per_warp";
    const int lh = P.lanes_per_hit;
    if (lh != 1 && lh != 2 && lh != 4 && lh != 8) return "lanes_per_hit must be 1, 2, 4 or 8";
    if (P.schedule < 0 || P.schedule > 2) return "schedule must be 0, 1 or 2";
    if (P.plain_per_sector < 0 || P.plain_per_sector > 2) return "plain_per_sector must be 0, 1 or 2";
    if (P.n_queues < 1 || P.n_queues > 64) return "n_queues must be in [1, 64]";
    if (P.refit != 0 && P.refit != 1) return "refit must be 0 or 1";
    if (P.merge != 0 && P.merge != 1) return "merge must be 0 or 1";
    if (P.merge && !P.refit) return "merge needs refit = 1 (it compares refitted states)";
    if (!(P.merge_chi2 > 0) || !(P.merge_gap > 0) || !(P.merge_overlap >= 0) || !(P.merge_window > 0))
        return "merge cuts must be positive";
    if (P.t0 != 0 && P.t0 != 1) return "t0 must be 0 or 1";
    if (P.count_work != 0 && P.count_work != 1) return "count_work must be 0 or 1";
    if (P.debug_wait_polls < 0) return "debug_wait_polls must be >= 0";
    if (P.t0 && !P.refit) return "t0 needs refit = 1 (it extrapolates refitted states)";
    if (!(P.t0_y_cut > 0) || !(P.t0_bin >= 0.01f) || !(P.t0_radius > 0) || P.t0_window < 0 || P.t0_n_min < 1)
        return "t0 parameters";
    for (int i = 0; i < 5; i++)
        if (!std::isfinite(P.field[i])) return "field terms must be finite";
    return nullptr;
}

extern "C" void tpc_params_default(tpc_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->k_win = 1.5f;
    p->d_max2 = 0.25f;
    p->l_seed = 3;
    p->sigma_y = 0.1f;
    p->sigma_z = 0.1f;
    p->var_s = 0.25f;
    p->var_q = 100.0f;
    p->var_t = 1.0f;
    p->n_sigma = 3.5f;
    p->w_min = 0.3f;
    p->w_max = 3.0f;
    p->s_max = 0.95f;
    p->y_margin = 2.0f;
    p->g_max = 8;
    p->n_min_tracklet = 10;
    p->n_min_track = 10;
    p->own_num = 7;
    p->own_den = 10;
    p->exact_fp32 = 0;
    p->bin_target = 1.0f;
    p->threads_per_row = 128;
    p->tracklets_per_warp = 32;
    p->lanes_per_hit = 1;
    p->plain_per_sector = 0;
    p->use_graph = 0;
    p->n_queues = 8;
    p->schedule = 2;
    p->refit = 0;
    p->merge = 0;
    p->merge_chi2 = 30.0f;
    p->merge_gap = 50.0f;
    p->merge_overlap = 5.0f;
    p->merge_window = 5.0f;
    p->t0 = 0;
    p->t0_y_cut = 1.0f;
    p->t0_bin = 0.25f;
    p->t0_radius = 1.0f;
    p->t0_window = 8;
    p->t0_n_min = 8;
    p->count_work = 0;
}

extern "C" int tpc_tracker_create(const tpc_geometry* g, double bz, const tpc_params* params,
                                  tpc_tracker** out)
{
    auto create_fail = [](const std::string& m) {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_create_err = m;
    };
    if (!g || !out) { create_fail("NULL geometry or output pointer"); return TPC_ERR_INVALID; }
    *out = nullptr;
    if (g->n_rows < 3 || g->n_rows > TPC_MAX_ROWS || !g->row_x) {
        create_fail("n_rows must be in [3, 256] with row_x given");
        return TPC_ERR_INVALID;
    }
    if (g->n_sectors < 2 || (g->n_sectors & 1)) { create_fail("n_sectors must be even and >= 2"); return TPC_ERR_INVALID; }
    for (int r = 0; r < g->n_rows; r++) {
        if (!(g->row_x[r] > 0) || !std::isfinite(g->row_x[r]) || (r && !(g->row_x[r] > g->row_x[r - 1]))) {
            create_fail("row_x must be finite, positive and strictly increasing");
            return TPC_ERR_INVALID;
        }
    }
    if (!(g->tan_half_open > 0) || !(g->z_max > 0) || !std::isfinite(bz)) {
        create_fail("tan_half_open, z_max must be > 0 and bz finite");
        return TPC_ERR_INVALID;
    }
    tpc_params P;
    tpc_params_default(&P);
    if (params) P = *params;
    if (const char* m = check_params(P)) { create_fail(std::string("params: ") + m); return TPC_ERR_INVALID; }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { create_fail("no CUDA device"); return TPC_ERR_DEVICE; }
    tpc_tracker* tr = new tpc_tracker();
    tr->dev = dev;
    tr->geom = *g;
    tr->row_x.assign(g->row_x, g->row_x + g->n_rows);
    tr->geom.row_x = tr->row_x.data();
    tr->bz = bz;
    tr->params = P;
    tr->kc = make_kconst(P, tr->geom, bz);
    cudaDeviceGetAttribute(&tr->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaStreamCreateWithFlags(&tr->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&tr->row_x_dev, sizeof(float) * TPC_MAX_ROWS) != cudaSuccess ||
        cudaMemcpy(tr->row_x_dev, tr->row_x.data(), sizeof(float) * g->n_rows,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMallocHost(&tr->counters_host, sizeof(int) * kNumCounters) != cudaSuccess) {
        create_fail("CUDA setup failed");
        tpc_tracker_destroy(tr);
        return TPC_ERR_DEVICE;
    }
    for (auto& e : tr->ev) cudaEventCreate(&e);
    *out = tr;
    return TPC_OK;
}

extern "C" void tpc_tracker_destroy(tpc_tracker* tr)
{
    if (!tr) return;
    cudaSetDevice(tr->dev);
    tpc_serve_shutdown(tr);
    if (tr->graph_exec) cudaGraphExecDestroy(tr->graph_exec);
    if (tr->own_stream) cudaStreamSynchronize(tr->own_stream);
    cudaFree(tr->ws);
    cudaFree(tr->row_x_dev);
    cudaFree(tr->dump_buf);
    cudaFreeHost(tr->counters_host);
    cudaFreeHost(tr->plan_host);
    for (auto& e : tr->ev) if (e) cudaEventDestroy(e);
    for (auto q : tr->queues) cudaStreamDestroy(q);
    for (auto e : tr->queue_ev) cudaEventDestroy(e);
    if (tr->fork_ev) cudaEventDestroy(tr->fork_ev);
    if (tr->own_stream) cudaStreamDestroy(tr->own_stream);
    delete tr;
}

extern "C" int tpc_tracker_set_params(tpc_tracker* tr, const tpc_params* params)
{
    if (!tr || !params) return TPC_ERR_INVALID;
    if (tpc_serve_busy(tr)) return tr->fail(TPC_BUSY, "stream tickets in flight");
    if (const char* m = check_params(*params)) return tr->fail(TPC_ERR_INVALID, std::string("params: ") + m);
    tr->params = *params;
    tr->kc = make_kconst(*params, tr->geom, tr->bz);
    tr->graph_key.clear();
    return TPC_OK;
}

extern "C" const char* tpc_last_error(const tpc_tracker* tr)
{
    if (!tr) {
        std::lock_guard<std::mutex> lk(g_err_mu);
        return g_create_err.c_str();
    }
    return tr->err.c_str();
}

// ------------------------------------------------------------- workspace

// Lay out every device buffer of one batch; returns the bytes needed.
size_t tpc_layout(const tpc_tracker* tr, const BatchShape& sh, DevPtrs* p, char* base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* r = base ? base + off : nullptr;
        off = align256(off + std::max<size_t>(bytes, 16));
        return r;
    };
    const size_t N = (size_t)sh.N, R = (size_t)sh.R, Tc = (size_t)sh.t_cap;
    const size_t NR = (size_t)tr->geom.n_rows;
    DevPtrs q{};
    q.clusters = reinterpret_cast<const float4*>(take(N * 16));
    // row_cnt, row_off and bin_cap_off are adjacent: one H2D of the host plan
    // fills all three
    q.row_cnt = reinterpret_cast<const int*>(take((3 * R + 2) * 4));
    q.row_off = q.row_cnt ? q.row_cnt + R : nullptr;
    q.bin_cap_off = q.row_off ? q.row_off + (R + 1) : nullptr;
    q.grid = reinterpret_cast<RowGrid*>(take(R * sizeof(RowGrid)));
    q.hits = reinterpret_cast<float4*>(take(N * 16));
    q.hyz = reinterpret_cast<float2*>(take((N + 2) * 8));  // + a pad entry read by whole-pair copies
    q.hpos = reinterpret_cast<int*>(take(N * 4));
    q.bin_off = reinterpret_cast<int*>(take((size_t)sh.bin_slots * 4));
    q.up = reinterpret_cast<int*>(take(N * 4));
    q.dn = reinterpret_cast<int*>(take(N * 4));
    q.up2 = reinterpret_cast<int*>(take(N * 4));
    q.dn2 = reinterpret_cast<int*>(take(N * 4));
    q.start_list = reinterpret_cast<int*>(take(N * 4));
    q.row_nstart = reinterpret_cast<int*>(take(R * 4));
    q.start_off = reinterpret_cast<int*>(take((R + 1) * 4));
    q.sched_off = reinterpret_cast<int*>(take((R + 1) * 4));
    q.start = reinterpret_cast<int*>(take(Tc * 4));
    q.t_row = reinterpret_cast<int*>(take(Tc * 4));
    q.t_state = reinterpret_cast<float4*>(take(Tc * 64));
    q.t_info = reinterpret_cast<int4*>(take(Tc * 16));
    q.sched = reinterpret_cast<int*>(take(Tc * 4));
    q.tl_f = reinterpret_cast<float*>(take(Tc * kTlFloats * 4));
    q.tl_n = reinterpret_cast<int*>(take(Tc * 4));
    q.tl_hits = reinterpret_cast<int*>(take(Tc * NR * 4));
    q.tl_work = reinterpret_cast<int4*>(take(Tc * 16));
    q.owner = reinterpret_cast<unsigned*>(take(N * 4));
    q.owned = reinterpret_cast<int*>(take(Tc * 4));
    q.acc = reinterpret_cast<int2*>(take(Tc * 8));
    q.acc_scan = reinterpret_cast<int2*>(take(Tc * 8));
    q.scan_part = reinterpret_cast<int2*>(take((Tc / kScanTile + 2) * 8));
    q.start_part = reinterpret_cast<int*>(take((R / kScanTile + 2) * 2 * 4));
    q.out_tracks = reinterpret_cast<tpc_track*>(take(Tc * sizeof(tpc_track)));
    q.out_hits = reinterpret_cast<int*>(take(N * 4));
    // the optional stages' buffers exist only when the stage is switched on
    const tpc_params& P = tr->params;
    auto opt = [&](bool on, size_t bytes) -> char* { return on ? take(bytes) : nullptr; };
    q.out_fits = reinterpret_cast<tpc_fit*>(opt(P.refit, Tc * sizeof(tpc_fit)));
    q.fit_bins = reinterpret_cast<int*>(opt(P.refit, 2 * (TPC_MAX_ROWS + 1) * 4));
    q.ev_first = reinterpret_cast<int2*>(take(((size_t)sh.n_events + 1) * 8));
    q.req_area = reinterpret_cast<int*>(take((size_t)sh.n_events * 4));
    q.out_merges = reinterpret_cast<tpc_merge*>(opt(P.merge, Tc * sizeof(tpc_merge)));
    q.mg_best = reinterpret_cast<unsigned long long*>(opt(P.merge, Tc * 16));
    q.unit_first = reinterpret_cast<int*>(opt(P.merge, ((size_t)sh.n_units + 1) * 4));
    q.mg_keys = reinterpret_cast<float2*>(opt(P.merge, Tc * 8));
    {
        const size_t E = (size_t)sh.n_events, nb = (size_t)std::max(tr->kc.t0_nb, 1);
        q.out_t0s = reinterpret_cast<tpc_t0*>(opt(P.t0, Tc * sizeof(tpc_t0)));
        q.t0_u = reinterpret_cast<float*>(opt(P.t0, Tc * 4));
        q.t0_bin = reinterpret_cast<int*>(opt(P.t0, Tc * 4));
        q.t0_hist = reinterpret_cast<int*>(opt(P.t0, E * nb * 4));
        q.t0_peak = reinterpret_cast<int*>(opt(P.t0, E * nb * 4));
        q.t0_npeak = reinterpret_cast<int*>(opt(P.t0, E * 4));
        q.t0_sum = reinterpret_cast<unsigned long long*>(opt(P.t0, E * nb * 8));
        q.t0_cnt = reinterpret_cast<int*>(opt(P.t0, E * nb * 4));
    }
    // set by the serving loop for its batches; the synchronous call does not rebase
    q.req_first_event = nullptr;
    q.counters = reinterpret_cast<int*>(take(kNumCounters * 4));
    q.N = sh.N;
    q.R = sh.R;
    q.n_units = sh.n_units;
    q.sched_block = 0;
    if (tr->params.schedule == 2 && sh.n_units > 0) {
        const double per_unit = std::max(1.0, (double)sh.N / sh.n_units);
        q.sched_block = (int)std::min<double>(sh.n_units, std::max(1.0, std::round(kSchedBlockClusters / per_unit)));
    }
    q.t_cap = sh.t_cap;
    q.m_cap = sh.t_cap;
    q.mh_cap = sh.N;
    if (p) *p = q;
    return off;
}

// The pinned plan buffer sized for a call of R rows.  Growing it means
// cudaFreeHost / cudaMallocHost, which synchronize the device: the request
// loop reserves a full batch's size when serving starts.
int tpc_reserve_plan(tpc_tracker* tr, int64_t R)
{
    if ((size_t)(3 * R + 2) <= tr->plan_cap) return TPC_OK;
    cudaFreeHost(tr->plan_host);
    tr->plan_host = nullptr;
    tr->plan_cap = 0;
    const size_t want = (size_t)(3 * R + 2) + (size_t)(R / 4) + 64;
    if (cudaMallocHost(&tr->plan_host, want * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return tr->fail(TPC_ERR_NOMEM, "cannot allocate pinned plan buffer");
    }
    tr->plan_cap = want;
    return TPC_OK;
}

// Shape of a batch from its (host) row counts.
int tpc_shape(tpc_tracker* tr, const int32_t* row_counts, int n_events, BatchShape* sh)
{
    const int NR = tr->geom.n_rows, S = tr->geom.n_sectors;
    const int64_t R = (int64_t)n_events * S * NR;
    if (R > (1 << 28)) return tr->fail(TPC_ERR_INVALID, "too many rows in one call");
    int64_t N = 0, bins = 0, max_unit = 0;
    int max_row = 0, max3 = 0, max_slots = 0, max_slots_nb = 0;
    const int rc_plan = tpc_reserve_plan(tr, R);
    if (rc_plan != TPC_OK) return rc_plan;
    // the pinned plan: row counts [R], CSR offsets of rows [R + 1], bin-table
    // offsets [R + 1], laid out as on the device so that one copy uploads all
    int* plan_cnt = tr->plan_host;
    int* plan_off = tr->plan_host + R;
    int* plan_bins = tr->plan_host + 2 * R + 1;
    if (plan_cnt != row_counts) std::memcpy(plan_cnt, row_counts, (size_t)R * sizeof(int));
    // bin-table slots per row count, for the current bin_target
    if (tr->slots_lut.size() != TPC_MAX_ROW_CLUSTERS + 1 || tr->slots_lut_bt != tr->params.bin_target) {
        tr->slots_lut.resize(TPC_MAX_ROW_CLUSTERS + 1);
        for (int c = 0; c <= TPC_MAX_ROW_CLUSTERS; c++)
            tr->slots_lut[(size_t)c] = row_bin_slots(c, tr->params.bin_target);
        tr->slots_lut_bt = tr->params.bin_target;
    }
    const int* lut = tr->slots_lut.data();
    for (int64_t u0 = 0; u0 < R; u0 += NR) {  // one (event, sector) unit at a time
        const int32_t* cnt = row_counts + u0;
        int ok = 1;
        for (int r = 0; r < NR; r++) ok &= (unsigned)cnt[r] <= (unsigned)TPC_MAX_ROW_CLUSTERS;
        if (!ok) {
            for (int r = 0; r < NR; r++) {
                if ((unsigned)cnt[r] > (unsigned)TPC_MAX_ROW_CLUSTERS) {
                    char m[128];
                    std::snprintf(m, sizeof m, "row_counts[%lld] = %d outside [0, %d]",
                                  (long long)(u0 + r), cnt[r], TPC_MAX_ROW_CLUSTERS);
                    return tr->fail(TPC_ERR_INVALID, m);
                }
            }
        }
        const int64_t n_before = N;
        for (int r = 0; r < NR; r++) {
            const int c = cnt[r];
            plan_off[u0 + r] = (int)N;
            plan_bins[u0 + r] = (int)bins;
            N += c;
            bins += lut[c];
            max_row = std::max(max_row, c);
            max_slots = std::max(max_slots, lut[c]);
        }
        max_unit = std::max<int64_t>(max_unit, N - n_before);
        for (int r = 1; r + 1 < NR; r++) {
            max3 = std::max(max3, cnt[r - 1] + cnt[r] + cnt[r + 1]);
            max_slots_nb = std::max(max_slots_nb, lut[cnt[r - 1]] + lut[cnt[r + 1]]);
        }
    }
    if (N >= (int64_t)1 << 30) return tr->fail(TPC_ERR_INVALID, "more than 2^30 clusters in one call");
    if (bins >= (int64_t)1 << 31) return tr->fail(TPC_ERR_INVALID, "search grid too large for one call");
    plan_off[R] = (int)N;
    plan_bins[R] = (int)bins;
    sh->n_events = n_events;
    sh->n_units = n_events * S;
    sh->R = (int)R;
    sh->N = (int)N;
    // cleaned links form disjoint chains with one start each, of >= l_seed hits
    sh->t_cap = (int)(N / std::max(2, tr->params.l_seed) + 1);
    sh->bin_slots = bins;
    sh->max_row = std::max(max_row, 1);
    sh->max3 = std::max(max3, 1);
    sh->max_unit = (int)max_unit;
    sh->max_slots = std::max(max_slots, 4);
    sh->max_slots_nb = std::max(max_slots_nb, 12);
    return TPC_OK;
}

int tpc_reserve(tpc_tracker* tr, size_t bytes)
{
    if (bytes <= tr->ws_bytes) return TPC_OK;
    if (tr->ws) {
        cudaStreamSynchronize(tr->own_stream);
        cudaDeviceSynchronize();
        cudaFree(tr->ws);
        tr->ws = nullptr;
        tr->ws_bytes = 0;
        tr->graph_key.clear();
    }
    size_t want = bytes + bytes / 4;
    if (cudaMalloc(&tr->ws, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&tr->ws, bytes) != cudaSuccess) {
            cudaGetLastError();
            tr->ws = nullptr;
            return tr->fail(TPC_ERR_NOMEM, "cannot allocate device workspace");
        }
        want = bytes;
    }
    tr->ws_bytes = want;
    return TPC_OK;
}

// --------------------------------------------------------------- pipeline

// Enqueue every device stage of one batch on stream s.  with_events records
// stage boundaries (not allowed while capturing a graph).
int tpc_enqueue(tpc_tracker* tr, const DevPtrs& p, const BatchShape& sh, cudaStream_t s,
                bool with_events)
{
    // Inside a stream capture, cudaEventRecordExternal adds a real
    // event-record node, so stage times are also available for graph replays
    // (a plain record would only become a dependency edge).
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    TPC_CUDA(cudaStreamIsCapturing(s, &cap_status));
    const unsigned rec_flags =
        cap_status == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
#define cudaEventRecord(ev_, s_) cudaEventRecordWithFlags(ev_, s_, rec_flags)
    const KConst& k = tr->kc;
    const tpc_params& P = tr->params;
    const float* xd = tr->row_x_dev;
    const bool exact = P.exact_fp32 != 0;
    auto nb = [&](const tpc::KConst& kk, const float* x, const DevPtrs& pp, int max3, int slots_nb, int th,
                  int u0, int nu, cudaStream_t ss) {
        const int lh = P.lanes_per_hit;
        return exact ? tpc_exact::launch_neighbours(kk, x, pp, max3, slots_nb, th, lh, u0, nu, ss)
                     : tpc_fast::launch_neighbours(kk, x, pp, max3, slots_nb, th, lh, u0, nu, ss);
    };
    auto seeds = [&](int u0, int u1, cudaStream_t ss) {
        return exact ? tpc_exact::launch_seeds(k, xd, p, tr->n_sm, u0, u1, ss)
                     : tpc_fast::launch_seeds(k, xd, p, tr->n_sm, u0, u1, ss);
    };
    auto tl = [&](int u0, int u1) {
        const int lpt = 32 / P.tracklets_per_warp;
        const bool cw = P.count_work != 0;
        return exact ? tpc_exact::launch_tracklets(k, xd, p, tr->n_sm, lpt, P.schedule, u0, u1, cw, s)
                     : tpc_fast::launch_tracklets(k, xd, p, tr->n_sm, lpt, P.schedule, u0, u1, cw, s);
    };
    const int th = P.threads_per_row;
    if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[0], s));
    TPC_CUDA(tpc_int::launch_plan(k, xd, p, tr->n_sm, s));
    if (!P.plain_per_sector) {
        TPC_CUDA(tpc_int::launch_grid(k, xd, p, sh.max_row, sh.max_slots, th, 0, sh.n_units, s));
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[1], s));
        TPC_CUDA(nb(k, xd, p, sh.max3, sh.max_slots_nb, th, 0, sh.n_units, s));
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[2], s));
        // the per-unit ownership kernel writes every owner key itself
        TPC_CUDA(tpc_int::launch_clean(k, p, th, 0, sh.n_units, false, s));
        TPC_CUDA(tpc_int::launch_start_scan(k, p, s));
        TPC_CUDA(tpc_int::launch_start_write(k, p, th, 0, sh.n_units, s));
        TPC_CUDA(seeds(0, sh.n_units, s));
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[3], s));
        TPC_CUDA(tl(-1, -1));
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[4], s));
        bool counted = false;
        TPC_CUDA(tpc_int::launch_owner_units(k, p, sh.n_units, sh.max_unit, tr->n_sm, s, &counted));
        TPC_CUDA(tpc_int::launch_select(k, p, tr->n_sm, 0, sh.n_units, false, s, counted));
    } else if (P.plain_per_sector == 2) {
        // Multi-queue scheme (Sec. 3.1, Fig. 3): each unit's stages in order
        // on one of n_queues streams, units round-robin; the two global steps
        // (start numbering, output compaction) join all queues.
        const int nq = P.n_queues;
        while ((int)tr->queues.size() < nq) {
            cudaStream_t q;
            cudaEvent_t e;
            TPC_CUDA(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
            TPC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            tr->queues.push_back(q);
            tr->queue_ev.push_back(e);
        }
        if (!tr->fork_ev) TPC_CUDA(cudaEventCreateWithFlags(&tr->fork_ev, cudaEventDisableTiming));
        auto fork = [&]() -> int {
            TPC_CUDA(cudaEventRecordWithFlags(tr->fork_ev, s, cudaEventRecordDefault));
            for (int q = 0; q < nq; q++) TPC_CUDA(cudaStreamWaitEvent(tr->queues[(size_t)q], tr->fork_ev, 0));
            return TPC_OK;
        };
        auto join = [&]() -> int {
            for (int q = 0; q < nq; q++) {
                TPC_CUDA(cudaEventRecordWithFlags(tr->queue_ev[(size_t)q], tr->queues[(size_t)q], 0));
                TPC_CUDA(cudaStreamWaitEvent(s, tr->queue_ev[(size_t)q], 0));
            }
            return TPC_OK;
        };
        int rc = fork();
        if (rc != TPC_OK) return rc;
        for (int u = 0; u < sh.n_units; u++) {
            cudaStream_t q = tr->queues[(size_t)(u % nq)];
            TPC_CUDA(tpc_int::launch_grid(k, xd, p, sh.max_row, sh.max_slots, th, u, 1, q));
            TPC_CUDA(nb(k, xd, p, sh.max3, sh.max_slots_nb, th, u, 1, q));
            TPC_CUDA(tpc_int::launch_clean(k, p, th, u, 1, true, q));
        }
        rc = join();
        if (rc != TPC_OK) return rc;
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[1], s));
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[2], s));
        TPC_CUDA(tpc_int::launch_start_scan(k, p, s));
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[3], s));
        rc = fork();
        if (rc != TPC_OK) return rc;
        for (int u = 0; u < sh.n_units; u++) {
            cudaStream_t q = tr->queues[(size_t)(u % nq)];
            TPC_CUDA(tpc_int::launch_start_write(k, p, th, u, 1, q));
            TPC_CUDA(seeds(u, u + 1, q));
            const int lpt = 32 / P.tracklets_per_warp;
            TPC_CUDA(exact ? tpc_exact::launch_tracklets(k, xd, p, tr->n_sm, lpt, P.schedule, u, u + 1, true, q)
                           : tpc_fast::launch_tracklets(k, xd, p, tr->n_sm, lpt, P.schedule, u, u + 1, true, q));
            TPC_CUDA(tpc_int::launch_select(k, p, tr->n_sm, u, u + 1, true, q));
        }
        rc = join();
        if (rc != TPC_OK) return rc;
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[4], s));
    } else {
        // The Run 1/2 scheduling (Sec. 3): every stage launched per sector.
        for (int u = 0; u < sh.n_units; u++)
            TPC_CUDA(tpc_int::launch_grid(k, xd, p, sh.max_row, sh.max_slots, th, u, 1, s));
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[1], s));
        for (int u = 0; u < sh.n_units; u++) TPC_CUDA(nb(k, xd, p, sh.max3, sh.max_slots_nb, th, u, 1, s));
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[2], s));
        for (int u = 0; u < sh.n_units; u++) TPC_CUDA(tpc_int::launch_clean(k, p, th, u, 1, true, s));
        TPC_CUDA(tpc_int::launch_start_scan(k, p, s));
        for (int u = 0; u < sh.n_units; u++) {
            TPC_CUDA(tpc_int::launch_start_write(k, p, th, u, 1, s));
            TPC_CUDA(seeds(u, u + 1, s));
        }
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[3], s));
        for (int u = 0; u < sh.n_units; u++) TPC_CUDA(tl(u, u + 1));
        if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[4], s));
        for (int u = 0; u < sh.n_units; u++)
            TPC_CUDA(tpc_int::launch_select(k, p, tr->n_sm, u, u + 1, true, s));
    }
    TPC_CUDA(tpc_int::launch_emit(k, p, tr->n_sm, s));
    if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[5], s));
    if (P.refit)
        TPC_CUDA(exact ? tpc_exact::launch_refit(k, p, tr->n_sm, s) : tpc_fast::launch_refit(k, p, tr->n_sm, s));
    if (P.merge)
        TPC_CUDA(exact ? tpc_exact::launch_merge(k, p, tr->n_sm, s) : tpc_fast::launch_merge(k, p, tr->n_sm, s));
    if (P.t0)
        TPC_CUDA(exact ? tpc_exact::launch_t0(k, p, tr->n_sm, sh.n_events, s)
                       : tpc_fast::launch_t0(k, p, tr->n_sm, sh.n_events, s));
    if (p.req_first_event) TPC_CUDA(tpc_int::launch_rebase(k, p, tr->n_sm, s));
    if (with_events) TPC_CUDA(cudaEventRecord(tr->ev[6], s));
#undef cudaEventRecord
    return TPC_OK;
}

static std::string graph_key_of(const tpc_tracker* tr, const BatchShape& sh, const DevPtrs& p)
{
    // every quantity a launch configuration (grid, shared memory, chunks,
    // kernel variant) is derived from
    char b[320];
    std::snprintf(b, sizeof b, "%d/%d/%d/%d/%d/%d/%d/%d/%p/%p/%d/%d/%d/%d/%d/%g/%d/%d", sh.N, sh.R,
                  sh.n_units, sh.max_row, sh.max3, sh.max_unit, sh.max_slots, sh.max_slots_nb,
                  (const void*)p.clusters, (const void*)p.counters,
                  tr->params.exact_fp32, tr->params.threads_per_row, tr->params.tracklets_per_warp,
                  tr->params.plain_per_sector, tr->params.schedule, (double)tr->params.bin_target,
                  tr->params.n_queues, tr->params.count_work);
    return std::string(b);
}

// Run all stages: directly, or as a replay of a captured graph when the
// batch shape and buffers match the captured ones.
int tpc_run_stages(tpc_tracker* tr, const DevPtrs& p, const BatchShape& sh, cudaStream_t s)
{
    if (!tr->params.use_graph) return tpc_enqueue(tr, p, sh, s, true);
    std::string key = graph_key_of(tr, sh, p);
    if (key != tr->graph_key) {
        if (tr->graph_exec) {
            cudaGraphExecDestroy(tr->graph_exec);
            tr->graph_exec = nullptr;
        }
        tr->graph_key.clear();
        cudaStream_t cs = tr->own_stream;
        TPC_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int rc = tpc_enqueue(tr, p, sh, cs, true);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (rc != TPC_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&tr->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return tr->fail(TPC_ERR_DEVICE, std::string("graph instantiate: ") + cudaGetErrorString(e));
        tr->graph_key = key;
    }
    TPC_CUDA(cudaGraphLaunch(tr->graph_exec, s));  // records the stage events itself
    return TPC_OK;
}

// The counters of the last call, read back to the host: checks the device
// error bits and keeps the result sizes.
static int check_counters(tpc_tracker* tr)
{
    const int* c = tr->counters_host;
    if (c[C_ERR] & E_INPUT) {
        int rr = c[C_BADROW] - 1;
        char m[160];
        int NR = tr->geom.n_rows, S = tr->geom.n_sectors;
        std::snprintf(m, sizeof m,
                      "invalid cluster (NaN/inf coordinate or x off its pad row) in event %d sector %d row %d",
                      rr / (NR * S), (rr / NR) % S, rr % NR);
        return tr->fail(TPC_ERR_INVALID, m);
    }
    if (c[C_ERR] & E_TIMEOUT) return tr->fail(TPC_ERR_TIMEOUT, "bulk copy wait ran out in a kernel");
    if (c[C_ERR] & E_SHAPE) return tr->fail(TPC_ERR_DEVICE, "a launch configuration did not fit the batch");
    tr->last_T = c[C_T];
    tr->last_M = c[C_M];
    tr->last_MH = c[C_MH];
    return TPC_OK;
}

// Enqueue the copies of tracks [t0, t1) and hits [h0, h1) of the device
// result into out (with the refit, merge and collision records of the same
// tracks when they are on and asked for).
static int enqueue_out(tpc_tracker* tr, const DevPtrs& p, tpc_output* out, int t0, int t1, int h0, int h1,
                       cudaStream_t s)
{
    const cudaMemcpyKind kind = out->mem_kind == TPC_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                : cudaMemcpyDeviceToHost;
    if (t1 > t0) {
        if (!out->tracks) return tr->fail(TPC_ERR_INVALID, "NULL tracks buffer");
        const size_t n = (size_t)(t1 - t0);
        TPC_CUDA(cudaMemcpyAsync(static_cast<tpc_track*>(out->tracks) + t0, p.out_tracks + t0,
                                 sizeof(tpc_track) * n, kind, s));
        if (out->fits && tr->params.refit)
            TPC_CUDA(cudaMemcpyAsync(static_cast<tpc_fit*>(out->fits) + t0, p.out_fits + t0,
                                     sizeof(tpc_fit) * n, kind, s));
        if (out->merges && tr->params.merge)
            TPC_CUDA(cudaMemcpyAsync(static_cast<tpc_merge*>(out->merges) + t0, p.out_merges + t0,
                                     sizeof(tpc_merge) * n, kind, s));
        if (out->t0s && tr->params.t0)
            TPC_CUDA(cudaMemcpyAsync(static_cast<tpc_t0*>(out->t0s) + t0, p.out_t0s + t0,
                                     sizeof(tpc_t0) * n, kind, s));
    }
    if (h1 > h0) {
        if (!out->hit_ids) return tr->fail(TPC_ERR_INVALID, "NULL hit_ids buffer");
        TPC_CUDA(cudaMemcpyAsync(static_cast<int*>(out->hit_ids) + h0, p.out_hits + h0,
                                 sizeof(int) * (size_t)(h1 - h0), kind, s));
    }
    return TPC_OK;
}

// Copy the device result into out, the part from track t_done and hit
// h_done on (the part before is there already), and wait for it.
static int copy_out_rest(tpc_tracker* tr, const DevPtrs& p, int M, int MH, tpc_output* out, cudaStream_t s,
                         int t_done, int h_done)
{
    if (!out) return tr->fail(TPC_ERR_INVALID, "NULL output");
    out->n_tracks = M;
    out->n_hits = MH;
    const int mt = std::min(M, std::max(out->cap_tracks, 0));
    const int mh = std::min(MH, std::max(out->cap_hits, 0));
    int rc = enqueue_out(tr, p, out, std::min(t_done, mt), mt, std::min(h_done, mh), mh, s);
    if (rc != TPC_OK) return rc;
    TPC_CUDA(cudaStreamSynchronize(s));
    if (mt < M || mh < MH) return tr->fail(TPC_ERR_OUTPUT_TRUNCATED, "output capacity too small");
    return TPC_OK;
}

// Copy the device result into out (the whole of it).
int tpc_copy_out(tpc_tracker* tr, const DevPtrs& p, int M, int MH, tpc_output* out, cudaStream_t s)
{
    return copy_out_rest(tr, p, M, MH, out, s, 0, 0);
}

extern "C" int tpc_track_sectors(tpc_tracker* tr, const tpc_cluster* clusters, const int32_t* row_counts,
                                 int n_events, int mem_kind, tpc_output* out, void* cuda_stream)
{
    if (!tr) return TPC_ERR_INVALID;
    if (!row_counts || n_events < 0 || !out) return tr->fail(TPC_ERR_INVALID, "NULL row_counts/out or n_events < 0");
    if (mem_kind != TPC_MEM_HOST && mem_kind != TPC_MEM_DEVICE) return tr->fail(TPC_ERR_INVALID, "mem_kind");
    TPC_CUDA(cudaSetDevice(tr->dev));
    BatchShape sh{};
    int rc = tpc_shape(tr, row_counts, n_events, &sh);
    if (rc != TPC_OK) return rc;
    if (sh.N > 0 && !clusters) return tr->fail(TPC_ERR_INVALID, "NULL clusters");
    if (mem_kind == TPC_MEM_DEVICE && (reinterpret_cast<uintptr_t>(clusters) & 15))
        return tr->fail(TPC_ERR_INVALID, "device clusters must be 16-byte aligned");
    cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : tr->own_stream;
    if (sh.n_units == 0 || sh.N == 0) {
        tr->last_T = tr->last_M = tr->last_MH = 0;
        tr->has_result = false;
        out->n_tracks = 0;
        out->n_hits = 0;
        return TPC_OK;
    }
    size_t bytes = tpc_layout(tr, sh, nullptr, nullptr);
    rc = tpc_reserve(tr, bytes);
    if (rc != TPC_OK) return rc;
    DevPtrs p;
    tpc_layout(tr, sh, &p, static_cast<char*>(tr->ws));
    if (mem_kind == TPC_MEM_HOST) {
        TPC_CUDA(cudaMemcpyAsync(const_cast<float4*>(p.clusters), clusters, (size_t)sh.N * 16,
                                 cudaMemcpyHostToDevice, s));
    } else {
        p.clusters = reinterpret_cast<const float4*>(clusters);
    }
    // row counts and the plan, from pinned memory in one copy
    TPC_CUDA(cudaMemcpyAsync(const_cast<int*>(p.row_cnt), tr->plan_host, (size_t)(3 * sh.R + 2) * 4,
                             cudaMemcpyHostToDevice, s));
    tr->cur = p;
    tr->cur_shape = sh;
    tr->has_result = false;
    tr->last_counted = tr->params.count_work != 0 || tr->params.plain_per_sector != 0;
    rc = tpc_run_stages(tr, p, sh, s);
    if (rc != TPC_OK) return rc;
    // Estimate first, fetch the rest if the estimate was short (Sec. 3.1):
    // the counters and the expected part of the output (the previous
    // result's size with a margin, within the capacities) go out together,
    // so that a result of the expected size takes one round trip to the
    // host.  Output entries past n_tracks / n_hits may be overwritten.
    const int est_t = std::min(std::max(out->cap_tracks, 0), tr->last_M + tr->last_M / 16 + 64);
    const int est_h = std::min(std::max(out->cap_hits, 0), tr->last_MH + tr->last_MH / 16 + 1024);
    TPC_CUDA(cudaMemcpyAsync(tr->counters_host, p.counters, sizeof(int) * kNumCounters, cudaMemcpyDeviceToHost, s));
    rc = enqueue_out(tr, p, out, 0, est_t, 0, est_h, s);
    if (rc != TPC_OK) return rc;
    TPC_CUDA(cudaStreamSynchronize(s));
    rc = check_counters(tr);
    if (rc != TPC_OK) return rc;
    tr->has_result = true;
    tr->last_stream = s;
    return copy_out_rest(tr, p, tr->last_M, tr->last_MH, out, s, est_t, est_h);
}

extern "C" int tpc_fetch_output(tpc_tracker* tr, tpc_output* out)
{
    if (!tr) return TPC_ERR_INVALID;
    if (!tr->has_result) return tr->fail(TPC_ERR_INVALID, "no result to fetch");
    TPC_CUDA(cudaSetDevice(tr->dev));
    return tpc_copy_out(tr, tr->cur, tr->last_M, tr->last_MH, out, tr->last_stream);
}

extern "C" int tpc_stage_times(tpc_tracker* tr, float* ms, int n)
{
    if (!tr || !ms) return TPC_ERR_INVALID;
    if (!tr->has_result) return tr->fail(TPC_ERR_INVALID, "no result");
    for (int i = 0; i < n && i < 7; i++) {
        float v = 0.0f;
        int a = i < 5 ? i : (i == 5 ? 0 : 5), b = i < 5 ? i + 1 : 6;
        if (cudaEventElapsedTime(&v, tr->ev[a], tr->ev[b]) != cudaSuccess) {
            cudaGetLastError();
            v = -1.0f;
        }
        ms[i] = v;
    }
    return TPC_OK;
}

extern "C" int tpc_debug_dump(tpc_tracker* tr, int what, void* dst, int64_t cap, int64_t* n_items)
{
    if (!tr || !dst || !n_items) return TPC_ERR_INVALID;
    if (!tr->has_result) return tr->fail(TPC_ERR_INVALID, "no result to dump");
    TPC_CUDA(cudaSetDevice(tr->dev));
    const DevPtrs& p = tr->cur;
    const int N = tr->cur_shape.N, T = tr->last_T, NR = tr->geom.n_rows;
    size_t bytes;
    switch (what) {
        case TPC_DUMP_LINKS_RAW:
        case TPC_DUMP_LINKS: *n_items = N; bytes = (size_t)N * 8; break;
        case TPC_DUMP_STARTS: *n_items = T; bytes = (size_t)T * 4; break;
        case TPC_DUMP_TRACKLETS: *n_items = T; bytes = (size_t)T * kTlFloats * 4; break;
        case TPC_DUMP_TRACKLET_N: *n_items = T; bytes = (size_t)T * 8; break;
        case TPC_DUMP_TRACKLET_HITS: *n_items = T; bytes = (size_t)T * NR * 4; break;
        case TPC_DUMP_TRACKLET_WORK:
            if (!tr->last_counted)
                return tr->fail(TPC_ERR_INVALID, "work counts need params.count_work = 1 in the call");
            *n_items = T;
            bytes = (size_t)T * 16;
            break;
        default: return tr->fail(TPC_ERR_INVALID, "unknown dump");
    }
    if ((int64_t)bytes > cap) return tr->fail(TPC_ERR_OUTPUT_TRUNCATED, "dump buffer too small");
    if (bytes == 0) return TPC_OK;
    cudaStream_t s = tr->own_stream;
    TPC_CUDA(cudaStreamSynchronize(tr->last_stream));
    if (bytes > tr->dump_bytes) {
        cudaFree(tr->dump_buf);
        tr->dump_buf = nullptr;
        tr->dump_bytes = 0;
        TPC_CUDA(cudaMalloc(&tr->dump_buf, bytes));
        tr->dump_bytes = bytes;
    }
    int* d = static_cast<int*>(tr->dump_buf);
    switch (what) {
        case TPC_DUMP_LINKS_RAW: TPC_CUDA(tpc_int::launch_dump_links(p, 0, d, s)); break;
        case TPC_DUMP_LINKS: TPC_CUDA(tpc_int::launch_dump_links(p, 1, d, s)); break;
        case TPC_DUMP_STARTS: TPC_CUDA(tpc_int::launch_dump_starts(p, T, d, s)); break;
        case TPC_DUMP_TRACKLETS:
            TPC_CUDA(cudaMemcpyAsync(d, p.tl_f, bytes, cudaMemcpyDeviceToDevice, s));
            break;
        case TPC_DUMP_TRACKLET_N:
            TPC_CUDA(cudaMemcpyAsync(d, p.tl_n, (size_t)T * 4, cudaMemcpyDeviceToDevice, s));
            TPC_CUDA(cudaMemcpyAsync(d + T, p.tl_n, (size_t)T * 4, cudaMemcpyDeviceToDevice, s));
            break;
        case TPC_DUMP_TRACKLET_HITS: TPC_CUDA(tpc_int::launch_dump_tl_hits(tr->kc, p, T, d, s)); break;
        case TPC_DUMP_TRACKLET_WORK: TPC_CUDA(tpc_int::launch_dump_tl_work(p, T, d, s)); break;
    }
    TPC_CUDA(cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, s));
    TPC_CUDA(cudaStreamSynchronize(s));
    if (what == TPC_DUMP_TRACKLET_N) {
        int* h = static_cast<int*>(dst);
        for (int t = 0; t < T; t++) h[T + t] = h[t] >= tr->params.n_min_tracklet ? 1 : 0;
    }
    return TPC_OK;
}

// ---------------------------------------------------------------- autotune

extern "C" int tpc_autotune(tpc_tracker* tr, const tpc_cluster* clusters, const int32_t* row_counts,
                            int n_events, int mem_kind, int reps, tpc_params* best, float* best_ms)
{
    if (!tr) return TPC_ERR_INVALID;
    if (tpc_serve_busy(tr)) return tr->fail(TPC_BUSY, "stream tickets in flight");
    if (reps < 1) reps = 3;
    tpc_output none{};  // capacity 0: the run completes, nothing is copied out
    auto run_ms = [&](float* ms) -> int {
        std::vector<float> v;
        for (int i = 0; i <= reps; i++) {  // the first run warms up (and captures a graph)
            none.tracks = nullptr;
            none.hit_ids = nullptr;
            none.cap_tracks = none.cap_hits = 0;
            none.mem_kind = TPC_MEM_HOST;
            int rc = tpc_track_sectors(tr, clusters, row_counts, n_events, mem_kind, &none, nullptr);
            if (rc != TPC_OK && rc != TPC_ERR_OUTPUT_TRUNCATED) return rc;
            float t = 0.0f;
            if (i > 0) {
                if (!tr->has_result || cudaEventElapsedTime(&t, tr->ev[0], tr->ev[5]) != cudaSuccess) {
                    cudaGetLastError();
                    return tr->fail(TPC_ERR_DEVICE, "autotune timing");
                }
                v.push_back(t);
            }
        }
        std::sort(v.begin(), v.end());
        *ms = v.empty() ? 0.0f : v[v.size() / 2];
        return TPC_OK;
    };
    tpc_params cur = tr->params;
    float cur_ms = 0.0f;
    int rc = run_ms(&cur_ms);
    if (rc != TPC_OK) return rc;
    struct Axis {
        int kind;  // 0 schedule, 1 bin_target, 2 tracklets_per_warp, 3 threads_per_row,
                   // 4 lanes_per_hit
        std::vector<float> values;
    };
    const std::vector<Axis> axes = {{0, {0, 1, 2}},
                                    {1, {0.25f, 0.5f, 1.0f, 2.0f}},
                                    {2, {32, 16, 8}},
                                    {3, {64, 128, 256}},
                                    {4, {1, 2, 4, 8}}};
    for (int pass = 0; pass < 2; pass++) {
        bool changed = false;
        for (const Axis& ax : axes) {
            for (float v : ax.values) {
                tpc_params cand = cur;
                if (ax.kind == 0) cand.schedule = (int)v;
                if (ax.kind == 1) cand.bin_target = v;
                if (ax.kind == 2) cand.tracklets_per_warp = (int)v;
                if (ax.kind == 3) cand.threads_per_row = (int)v;
                if (ax.kind == 4) cand.lanes_per_hit = (int)v;
                if (std::memcmp(&cand, &cur, sizeof cand) == 0) continue;
                rc = tpc_tracker_set_params(tr, &cand);
                if (rc != TPC_OK) return rc;
                float ms = 0.0f;
                rc = run_ms(&ms);
                if (rc != TPC_OK) return rc;
                if (ms < cur_ms * 0.99f) {
                    cur = cand;
                    cur_ms = ms;
                    changed = true;
                }
            }
            rc = tpc_tracker_set_params(tr, &cur);
            if (rc != TPC_OK) return rc;
        }
        if (!changed) break;
    }
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return TPC_OK;
}
