// dcsc.cu -- column-block DCSC tiles (placeholder until the tiled kernels land).
#include "bfs_internal.h"

namespace bfsrt {

bfs_status build_dcsc_tiles(bfs_graph*, cudaStream_t) {
    return fail(BFS_ERR_UNSUPPORTED, "DCSC tiles are not built yet");
}

}  // namespace bfsrt
