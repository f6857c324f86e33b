// gke_split.h -- split-precision (BF16 x3) tensor-core correlator: workspace
// and entry points used by the plan (internal).
#pragma once
#include <cuda_runtime.h>
#include <string>
#include "../../include/gke.h"
#include "gke_common.cuh"

namespace gke {

struct SplitWork {
    void* ops = nullptr;        // BF16 slice operands (A blocks, then B blocks)
    size_t ops_bytes = 0, a_bytes = 0, b_bytes = 0;
    int* err = nullptr;         // device flag: a pipeline wait timed out
};

gke_status split_alloc(SplitWork& w, int ny, int ns, int Kc);
cudaError_t split_setup(cudaStream_t st);
gke_status split_correlate(SplitWork& w, const zf* Xop, int ns, int ny, int Nk, int k0, int Kc, zf* raw,
                           unsigned jobs, cudaStream_t st, std::string& err, int* launches);
gke_status split_check(SplitWork& w, cudaStream_t st, std::string& err);
void split_free(SplitWork& w);

}  // namespace gke
