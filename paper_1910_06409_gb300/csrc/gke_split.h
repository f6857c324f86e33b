// gke_split.h -- split-precision (BF16 x3) tensor-core correlator: workspace
// and entry points used by the plan (internal).
#pragma once
#include <cuda_runtime.h>
#include <string>
#include "../../include/gke.h"
#include "gke_common.cuh"

namespace gke {

struct SplitWork {
    void* ops = nullptr;        // split operand planes
    size_t ops_bytes = 0;
};

gke_status split_alloc(SplitWork& w, int ny, int ns, int Nk);
cudaError_t split_setup(cudaStream_t st);
gke_status split_correlate(SplitWork& w, const zd* Xop, int ns, int ny, int Nk, int beta, zd* acc_sq, zd* acc_D,
                           cudaStream_t st, std::string& err, int* launches);
void split_free(SplitWork& w);

}  // namespace gke
