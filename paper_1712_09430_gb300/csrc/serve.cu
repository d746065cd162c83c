// Request loop (continuous batching): placeholder until the serving path lands.
#include "tpc_serve.h"

struct ServeState {};

void tpc_serve_shutdown(tpc_tracker* tr) { (void)tr; }
bool tpc_serve_busy(const tpc_tracker* tr) { (void)tr; return false; }

extern "C" int tpc_stream_submit(tpc_tracker* tr, const tpc_cluster*, const int32_t*, int, uint64_t,
                                 uint64_t*)
{
    if (!tr) return TPC_ERR_INVALID;
    return tr->fail(TPC_ERR_INVALID, "serving not available");
}

extern "C" int tpc_stream_poll(tpc_tracker* tr, uint64_t, tpc_output*, int)
{
    if (!tr) return TPC_ERR_INVALID;
    return tr->fail(TPC_ERR_INVALID, "serving not available");
}
