// bfs_multi.cu -- batched multi-source BFS (placeholder until the lane-mask kernels land).
#include "bfs_internal.h"

namespace bfsrt {

bfs_status multi_prepare(bfs_graph*, cudaStream_t) { return fail(BFS_ERR_UNSUPPORTED, "bfs_run_multi: not built yet"); }
bfs_status multi_launch(bfs_graph*, const int32_t*, int32_t, int32_t*, int32_t*, const bfs_options&, cudaStream_t) {
    return fail(BFS_ERR_UNSUPPORTED, "bfs_run_multi: not built yet");
}
bfs_status multi_collect_status(bfs_graph*, cudaStream_t) { return BFS_OK; }
void multi_release(bfs_graph*) {}
bfs_status build_dcsc_tiles(bfs_graph*, cudaStream_t) { return fail(BFS_ERR_UNSUPPORTED, "DCSC tiles: not built yet"); }

}  // namespace bfsrt
