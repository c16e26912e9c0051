// Batched and served queries (placeholder entry points until the lane kernels land).
#include "rpq_internal.h"

using namespace rpq;

extern "C" rpq_status rpq_serve_create(const rpq_graph *, const rpq_serve_config *, rpq_server **) {
    return fail(RPQ_ERR_INVALID, "serving is not available in this build");
}
extern "C" rpq_status rpq_serve_submit(rpq_server *, const rpq_nfa *, int32_t, uint64_t *) {
    return fail(RPQ_ERR_INVALID, "serving is not available in this build");
}
extern "C" rpq_status rpq_serve_poll(rpq_server *, uint64_t, int32_t *, int64_t, int64_t *) {
    return fail(RPQ_ERR_INVALID, "serving is not available in this build");
}
extern "C" rpq_status rpq_serve_drain(rpq_server *, int64_t) {
    return fail(RPQ_ERR_INVALID, "serving is not available in this build");
}
extern "C" rpq_status rpq_serve_stats_get(rpq_server *, rpq_serve_stats *) {
    return fail(RPQ_ERR_INVALID, "serving is not available in this build");
}
extern "C" void rpq_serve_destroy(rpq_server *) {}
