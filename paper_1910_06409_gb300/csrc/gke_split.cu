// gke_split.cu -- split-precision correlator (placeholder until the tcgen05
// kernel lands): reports GKE_ERR_UNSUPPORTED.
#include "gke_split.h"

namespace gke {

gke_status split_alloc(SplitWork& w, int, int, int) { w.ops = nullptr; w.ops_bytes = 0; return GKE_OK; }
cudaError_t split_setup(cudaStream_t) { return cudaSuccess; }
gke_status split_correlate(SplitWork&, const zd*, int, int, int, int, zd*, zd*, cudaStream_t, std::string& err, int* launches)
{
    *launches = 0;
    err = "split-precision correlator not available in this build";
    return GKE_ERR_UNSUPPORTED;
}
void split_free(SplitWork& w) { w.ops = nullptr; }

}  // namespace gke
