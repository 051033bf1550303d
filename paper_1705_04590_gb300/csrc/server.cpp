// server.cpp -- placeholder until the continuous-batching server lands.
#include "bfs_internal.h"

using namespace bfsrt;

extern "C" {
bfs_status bfs_server_create(int64_t, int32_t, bfs_server** out) {
    if (out) *out = nullptr;
    return fail(BFS_ERR_UNSUPPORTED, "server: not built yet");
}
bfs_status bfs_server_add_graph(bfs_server*, bfs_graph*, int32_t*) { return fail(BFS_ERR_UNSUPPORTED, "server"); }
bfs_status bfs_submit(bfs_server*, int32_t, int32_t, int32_t*, uint64_t*) { return fail(BFS_ERR_UNSUPPORTED, "server"); }
bfs_status bfs_poll(bfs_server*, uint64_t) { return fail(BFS_ERR_UNSUPPORTED, "server"); }
bfs_status bfs_wait(bfs_server*, uint64_t, int64_t) { return fail(BFS_ERR_UNSUPPORTED, "server"); }
bfs_status bfs_server_stats(bfs_server*, int64_t*) { return fail(BFS_ERR_UNSUPPORTED, "server"); }
bfs_status bfs_ticket_latency_us(bfs_server*, uint64_t, double*) { return fail(BFS_ERR_UNSUPPORTED, "server"); }
void bfs_server_destroy(bfs_server*) {}
}
