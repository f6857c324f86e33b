// gke_kernels.h -- internal declarations shared by the .cu files of the
// library (not part of the public C ABI, which is include/gke.h).
#pragma once
#include <cuda_runtime.h>
#include "gke_common.cuh"

namespace gke {

// rows of the device profile array prof[NPR][ny]
enum Prof { PR_U = 0, PR_V, PR_W, PR_P, PR_DU, PR_EPS, PR_Q, PR_UV, PR_PV, PR_QU, PR_QV, PR_QW, NPR };

struct PairCoef { double dU, Upm, dUp, nu, inv_count; };

void upload_jobs(cudaStream_t st);

__global__ void k_mean_accum(const zd* fields, int ns, int ny, long long plane, double* mean_sum);
__global__ void k_load_linear(const zd* fields, int ns, int ny, int Nk, const double* mean, zd* Xop,
                              int* nonfinite);
__global__ void k_col_inverse(const zd* fields_s, int ny, int nz, int nxh, int CW, const double* mean,
                              const zd* tw_z, zd* G);
__global__ void k_row_products(const zd* G, int ny, int nz, int nx, int RZ, const zd* tw_x, zd* H,
                               double* part);
__global__ void k_col_forward(const zd* H, int ny, int nz, int nxh, int CW, int YB, int s, int ns,
                              const zd* tw_z, zd* Xop);
__global__ void k_eps(const zd* Xop, int ns, int ny, int nz, int nxh, int nx, double Lx, double Lz,
                      const double* fdw, const int* fdl0, int kchunk, double* part);
__global__ void k_reduce_partials(const double* part, int nvals, int nb, double* out);
__global__ void k_correlate_f64(const zd* Xop, int ns, int ny, int Nk, int beta, zd* acc_sq, zd* acc_D);
__global__ void k_terms_colpass(const zd* acc_sq, const zd* acc_D, const int* pair_i, long long pair0,
                                int ny, int nz, int nx, int CW, double Lx, double Lz, double nu,
                                double inv_count, const double* prof, const zd* tw_z, zd* W);
__global__ void k_terms_rowpass(const zd* W, const int* pair_i, long long pair0, long long npair, int ny,
                                int nz, int nx, int RZ, const double* prof, const zd* tw_x, double* terms);
__global__ void k_stencil_A(double* terms, long long npair, const int* pair_i, int ny, int nz, int nx,
                            double nu, const double* fdw, const int* fdl0);
__global__ void k_stencil_res(double* terms, long long npair, const int* pair_i, int ny, int nz, int nx,
                              const double* fdw, const int* fdl0);
__global__ void k_profiles(const double* mean_sum, double mean_count, const double* stats,
                           double snap_count, long long plane_points, double nu, const double* fdw,
                           const int* fdl0, int ny, double* prof);

}  // namespace gke
