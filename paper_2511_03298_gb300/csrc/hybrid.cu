// Hybrid intra-cluster search (Sec. 4.4): per-list 32-NN graphs.
#include "index.cuh"

namespace ksc {
int build_graph(ksc_index* ix, cudaStream_t st) {
    (void)ix;
    (void)st;
    ksc::set_error("graph construction is not available in this build");
    return KSC_EUNSUPPORTED;
}
}  // namespace ksc
