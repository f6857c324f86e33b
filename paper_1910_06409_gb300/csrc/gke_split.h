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
// plane mode: grids whose wall-normal rows fit four 128-row tiles (ny <= 512
// or ny = 513); the plane spectra of wavenumbers [k0, k0 + Kc) into
// out[NPLANE][Kc][npp], npp >= npair a multiple of 4 (planes: bit j = Plane j)
bool split_planes_ok(int ny);
gke_status split_correlate_planes(SplitWork& w, const zf* Xop, int ns, int ny, int Nk, int k0, int Kc,
                                  unsigned planes, long long npp, const double* prof, zf* out, cudaStream_t st,
                                  std::string& err, int* launches);
gke_status split_check(SplitWork& w, cudaStream_t st, std::string& err);
void split_free(SplitWork& w);

}  // namespace gke
