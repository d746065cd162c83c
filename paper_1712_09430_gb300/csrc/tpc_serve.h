// Host-internal state of a tracker and the request loop (continuous batching).
#pragma once
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "tpc_dev.cuh"

struct BatchShape {
    int n_events = 0, n_units = 0, R = 0, N = 0, t_cap = 0;
    int64_t bin_slots = 0;
    int max_row = 1, max3 = 1;
    int max_unit = 0;  // clusters of the largest (event, sector) unit
    // bin-table slots of the largest row, and of the largest pair of rows
    // r - 1 and r + 1 (shared memory of the grid and neighbour kernels)
    int max_slots = 4, max_slots_nb = 12;
};

struct ServeState;  // defined in serve.cu

struct tpc_tracker {
    int dev = 0;
    int n_sm = 0;
    tpc_geometry geom{};
    std::vector<float> row_x;
    double bz = 0.0;
    tpc_params params{};
    tpc::KConst kc{};
    float* row_x_dev = nullptr;
    cudaStream_t own_stream = nullptr;
    // workspace of synchronous calls
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // last synchronous call
    tpc::DevPtrs cur{};
    BatchShape cur_shape{};
    bool has_result = false;
    bool last_counted = false;     // the last call's constructor counted its work
    int last_T = 0, last_M = 0, last_MH = 0;
    cudaStream_t last_stream = nullptr;
    int* counters_host = nullptr;  // pinned
    int* plan_host = nullptr;      // pinned: row counts, row CSR offsets, bin-table offsets of a call
    size_t plan_cap = 0;           // ints
    std::vector<int> slots_lut;    // bin-table slots per row count (current bin_target)
    float slots_lut_bt = 0.0f;
    cudaEvent_t ev[7] = {};
    // graph replay of the batched stages
    cudaGraphExec_t graph_exec = nullptr;
    std::string graph_key;
    // multi-queue per-sector form: streams and fork/join events
    std::vector<cudaStream_t> queues;
    std::vector<cudaEvent_t> queue_ev;
    cudaEvent_t fork_ev = nullptr;
    // debug dumps
    void* dump_buf = nullptr;
    size_t dump_bytes = 0;
    // serving
    ServeState* serve = nullptr;
    std::string err;

    int fail(int code, const std::string& msg);
};

// tracker.cu
size_t tpc_layout(const tpc_tracker* tr, const BatchShape& sh, tpc::DevPtrs* p, char* base);
int tpc_shape(tpc_tracker* tr, const int32_t* row_counts, int n_events, BatchShape* sh);
int tpc_reserve_plan(tpc_tracker* tr, int64_t R);
int tpc_enqueue(tpc_tracker* tr, const tpc::DevPtrs& p, const BatchShape& sh, cudaStream_t s,
                bool with_events);

// serve.cu
void tpc_serve_shutdown(tpc_tracker* tr);
bool tpc_serve_busy(const tpc_tracker* tr);
