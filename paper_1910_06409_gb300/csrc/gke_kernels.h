// gke_kernels.h -- internal declarations shared by the .cu files of the
// library (not part of the public C ABI, which is include/gke.h).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <algorithm>

#include "gke_common.cuh"

namespace gke {

// rows of the device profile array prof[NPR][ny]
enum Prof { PR_U = 0, PR_V, PR_W, PR_P, PR_DU, PR_EPS, PR_Q, PR_UV, PR_PV, PR_QU, PR_QV, PR_QW, NPR };

void upload_jobs(cudaStream_t st);

// Terms a request expands to: Phi_y and phi carry the Step-3 FD parts of A
// (Eq. 10-11); the residual takes Y1 / Y2 derivatives of Phi_y and phi.
inline unsigned term_set(unsigned m)
{
    const unsigned all = (1u << NTERM) - 1u;
    m = m ? (m & all) : all;
    if (m & (1u << T_RES)) m |= (1u << T_PHIY) | (1u << T_PHI);
    if (m & ((1u << T_PHIY) | (1u << T_PHI))) m |= 1u << T_A;
    return m;
}

// Contractions (bit j = job j) the spectra of a term set combine
// (k_combine: A = -2 S0, Phi_x from Gx and D, Phi_y from QV and X2, Phi_z from
// Gz and D, phi from QV, X2 and F, xi from E, the residual from Gx, Gz, D, E)
inline unsigned job_set(unsigned t)
{
    auto b = [](int j) { return 1u << j; };
    unsigned j = 0;
    if (t & (1u << T_A)) j |= b(J_D);
    if (t & (1u << T_PHIX)) j |= b(J_GX) | b(J_D);
    if (t & (1u << T_PHIY)) j |= b(J_QV) | b(J_X);
    if (t & (1u << T_PHIZ)) j |= b(J_GZ) | b(J_D);
    if (t & (1u << T_PHI)) j |= b(J_QV) | b(J_X) | b(J_F);
    if (t & (1u << T_XI)) j |= b(J_E);
    if (t & (1u << T_RES)) j |= b(J_GX) | b(J_GZ) | b(J_D) | b(J_E);
    return j;
}

// Planes (bit j = Plane j) the spectra of a term set are formed from:
// A = A; Phi_x = S4 + (dU - 2 i nu kx) A; Phi_y; Phi_z = S6 - 2 i nu kz A;
// phi; xi; residual = i kx Phi_x + i kz Phi_z - xi
inline unsigned plane_set(unsigned t)
{
    auto b = [](int j) { return 1u << j; };
    unsigned p = 0;
    if (t & ((1u << T_A) | (1u << T_PHIX) | (1u << T_PHIZ) | (1u << T_RES))) p |= b(PL_A);
    if (t & ((1u << T_PHIX) | (1u << T_RES))) p |= b(PL_S4);
    if (t & (1u << T_PHIY)) p |= b(PL_PHIY);
    if (t & ((1u << T_PHIZ) | (1u << T_RES))) p |= b(PL_S6);
    if (t & (1u << T_PHI)) p |= b(PL_PHI);
    if (t & ((1u << T_XI) | (1u << T_RES))) p |= b(PL_XI);
    return p;
}

// the n-th set bit of m (n < popcount(m))
__host__ __device__ __forceinline__ int nth_bit(unsigned m, int n)
{
    for (int i = 0; i < 32; ++i)
        if ((m >> i) & 1u) { if (n == 0) return i; --n; }
    return -1;
}
// Transform tile parameters for a grid and a complex size (bytes): each CTA
// keeps its ping-pong buffers and twiddles within 64 KB, so three CTAs fit
// on an SM.  The plan and the allocation-free entry point both use these.
struct Tiles { int cw_ci, rz_rp, cw_cf, yb_cf, cw_tc, rz_tr; };
inline Tiles pick_tiles(int nx, int nz, size_t csz)
{
    Tiles t;
    const size_t lim = 64 * 1024;
    auto fits = [&](size_t elems) { return elems * csz <= lim; };
    t.cw_ci = 16; while (t.cw_ci > 1 && !fits((size_t)(1 + 2 * t.cw_ci) * nz)) t.cw_ci /= 2;
    t.rz_rp = 8;  while (t.rz_rp > 1 && !fits((size_t)(1 + 8 * t.rz_rp) * nx)) t.rz_rp /= 2;
    t.cw_cf = 4; t.yb_cf = 8;
    while (t.cw_cf * t.yb_cf > 1 && !fits((size_t)(1 + 2 * t.cw_cf * t.yb_cf) * nz)) {
        if (t.cw_cf > 1) t.cw_cf /= 2; else t.yb_cf /= 2;
    }
    t.cw_tc = 16; while (t.cw_tc > 1 && !fits((size_t)(1 + 2 * t.cw_tc) * nz)) t.cw_tc /= 2;
    t.rz_tr = 8;  while (t.rz_tr > 1 && !fits((size_t)(1 + 8 * t.rz_tr) * nx)) t.rz_tr /= 2;
    return t;
}
// wavenumbers per CTA of the dissipation sums, and the doubles of the
// partial-sum buffer of the products stage (row sums of the row passes,
// then the dissipation chunks)
constexpr int EPS_KCHUNK = 16;
inline size_t part_count(int nz, int ny, int Nk, const Tiles& t)
{
    const size_t rows = (size_t)6 * ny * std::max((nz + t.rz_rp - 1) / t.rz_rp, (nz + 3) / 4);
    const size_t eps = (size_t)ny * ((Nk + EPS_KCHUNK - 1) / EPS_KCHUNK);
    return std::max(rows, eps);
}
// transform lengths of the Stockham kernels: 2^a or 3 * 2^a
inline bool fft_len_ok(int n)
{
    auto pow2 = [](int m) { return m > 0 && (m & (m - 1)) == 0; };
    return pow2(n) || (n % 3 == 0 && pow2(n / 3));
}

int combine_kc(bool fp32);
bool combine_kc_ok(bool fp32, int kc);

__global__ void k_mean_accum(const zd* fields, int ns, int ny, long long plane, double* mean_sum);
__global__ void k_reduce_partials(const double* part, int nvals, int nb, double* out);
void correlate_launch(bool fp32, const void* Xop, int ns, int ny, int Nk, int k0, int Kc, void* raw, unsigned jobs,
                      cudaStream_t st);

// products stage (gke_products.cu); complex<TF> buffers passed as void*
struct ProdArgs {
    const zd* fields; int ns, ny, nz, nx, nxh, Nk;
    const double* mean; void* Xop; void* G; void* H; const void* tw_x; const void* tw_z;
    double* part; double* stats; int* nonfinite;
    int cw_ci, rz_rp, cw_cf, yb_cf, eps_kchunk;
    double Lx, Lz; const double* fdw; const int* fdl0;
    cudaStream_t st;
    // optional second stream and buffers: odd snapshots run there
    cudaStream_t st2 = nullptr;
    void* G2 = nullptr; void* H2 = nullptr; double* part2 = nullptr;
    const cudaEvent_t* ev = nullptr;      // 6 caller-owned events for st2 (else created per call)
    // optional: event s completes when snapshot s of `fields` has arrived on
    // the device; each snapshot's linear operands and transforms wait for it
    const cudaEvent_t* up_ev = nullptr;
};
template <typename TF> int products_launch(const ProdArgs& a);
cudaError_t products_set_attrs(int lim);

// term spectra (gke_combine.cu)
int combine_launch(bool fp32_in, bool out64, const void* raw, int ny, int nz, int nx, double Lx, double Lz,
                   double nu, const double* prof, int beta, int kbase, int Kc, long long cstride, void* comb,
                   unsigned terms, int kc, cudaStream_t st);
// chunked mode: the chunk's wavenumber rows gathered into a contiguous
// operand set, and the fused combine + aliasing fold of its contractions into
// the FP64 coarse spectra of every triangle pair (rows: the chunk's kz rows,
// crs: the coarse rows they complete)
int gather_rows_launch(bool c64, const void* src, int nf, long long Nk, long long per_k, const int* rows, int nrows,
                       int nxh, void* dst, cudaStream_t st);
// Step 1 for velocity-vorticity databases (gke_step1.cu): the band storage
// of the factored Poisson operators, shared-memory attributes, the
// factorisation (once per plan) and the five kernels of one snapshot
size_t s1_band_doubles(int ny, long long Nk);
cudaError_t s1_set_attrs(int nx, int nz);
int s1_factor_launch(int ny, int nz, int nx, double Lx, double Lz, const double* w1, const double* w2, const int* l0,
                     double* ab, unsigned char* piv, cudaStream_t st);
int s1_snapshot_launch(const zd* v_eta, const double* mean_uw, int ny, int nz, int nx, double Lx, double Lz,
                       double nu, const double* w1, const double* w2, const int* l0, const zd* tw_x, const zd* tw_z,
                       const double* ab, const unsigned char* piv, zd* bufA, zd* bufB, zd* out, cudaStream_t st);
int planes_fold_launch(const void* planes, long long npp, int Kc, const int* rows, int nrows, const int* crs, int ncr,
                       const int* pair_tri, long long npair, int ny, int nz, int nx, int nzd, int nxd, double Lx,
                       double Lz, double nu, const double* prof, unsigned tmask, void* dec, cudaStream_t st);
int combine_fold_launch(bool c64, const void* raw, const int* rows, int nrows, const int* crs, int ncr, int ny,
                        int nz, int nx, int nzd, int nxd, double Lx, double Lz, double nu, const double* prof,
                        unsigned tmask, void* dec, cudaStream_t st);
int promote_launch(const void* comb32, long long n, void* comb64, cudaStream_t st);
int planes_accum_launch(const void* src, long long per_plane, unsigned planes, int beta, void* dst, cudaStream_t st);
int mirror_fold_launch(bool c64, const void* comb, const int* pair_w, long long nout, int ny, int Nk, void* out,
                       cudaStream_t st);
cudaError_t combine_set_attrs();

// Separations kept in the output (a-posteriori undersampling, Sec. 3.4):
// nrz rows and nrx columns of the nz x nx separation grid.  NULL tables mean
// full resolution.
struct SepMap {
    int nz, nx, nrz, nrx;
    const int* zpos;      // [nz]: kept row of separation index m_z, or -1
    const int* xpos;      // [nx]: kept column of m_x, or -1
    const int* negz;      // [nrz]: kept row of -r_z (the kept set is symmetric)
    const int* negx;      // [nrx]: kept column of -r_x
    __device__ __forceinline__ int zrow(int z) const { return zpos ? zpos[z] : z; }
    __device__ __forceinline__ int xcol(int x) const { return xpos ? xpos[x] : x; }
    __device__ __forceinline__ int zneg(int zr) const { return negz ? negz[zr] : (nz - zr) % nz; }
    __device__ __forceinline__ int xneg(int xr) const { return negx ? negx[xr] : (nx - xr) % nx; }
};

inline SepMap full_sep(int nz, int nx)
{
    SepMap m;
    m.nz = m.nrz = nz;
    m.nx = m.nrx = nx;
    m.zpos = m.xpos = m.negz = m.negx = nullptr;
    return m;
}

// inverse transforms (gke_terms.cu)
struct TermArgs {
    bool fp32;            // split path: FP32 transforms and FP32 terms
    bool comb64;          // comb holds complex128 (else complex64)
    const void* comb; void* W; const int* pair_i; long long npair, pair_chunk;
    int ny, nz, nx, cw, rz; double inv_count; const double* prof; const void* tw_x; const void* tw_z;
    void* terms; float* spec; SepMap sep; cudaStream_t st;
    unsigned tmask = (1u << NTERM) - 1u;  // terms to transform (term_set)
    // optional: a second stream and scratch buffer (column and row passes of
    // successive chunks overlap); a callback after the launches of each pair
    // chunk [p0, p0 + np), given the stream its row pass ran on
    cudaStream_t st2 = nullptr;
    void* W2 = nullptr;
    const cudaEvent_t* ev = nullptr;      // 4 caller-owned events for st2 (else created per call)
    void (*after_chunk)(void* ctx, long long p0, long long np, cudaStream_t st) = nullptr;
    void* ctx = nullptr;
    // split plane mode: the column pass forms the terms from the plane spectra
    // planes[NPLANE][Kc][npp] (complex128 if planes64, else complex64)
    // instead of reading comb; pair chunks are multiples of 4
    const void* planes = nullptr;
    bool planes64 = false;
    long long npp = 0;
    int Kc = 0;
    double Lx = 0, Lz = 0, nu = 0;
};
int terms_launch(const TermArgs& a);
cudaError_t terms_set_attrs(int lim);
int stencil_launch(bool fp32, int wedge, void* terms, float* spec, long long npair, const int* pair_i, int ny,
                   const SepMap& sep, double nu, const double* fdw, const int* fdl0, const double* prof,
                   unsigned tmask, cudaStream_t st);

__global__ void k_freeze_mean(double* mean_sum, double mean_count, int mirror, int ny, double* mean);
__global__ void k_profiles(const double* mean_sum, double mean_count, const double* stats,
                           double snap_count, long long plane_points, double nu, int mirror, const double* fdw,
                           const int* fdl0, int ny, double* prof);

}  // namespace gke
