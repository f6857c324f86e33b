// gke1h.cu -- the GKE for a flow with one homogeneous direction (x): plan,
// kernels and the C ABI of include/gke1h.h.
//
// The paper's method (Sec. 3) with Parseval in x only and the second
// inhomogeneous direction z handled like the wall-normal one (Sec. 5): every
// pair of cross-section points (p1, p2) plays the part of a (Y1, Y2) pair.
// Stages of one evaluation (FP64 plans; FP32 plans as noted at the end):
//   mean       k1_mean: U_f(p), the m_x = 0 coefficient averaged over the
//              snapshots (Step 1); k1_grad: d_y U_i, d_z U_i by the stencils.
//   products   k1_products, one CTA per point p: per snapshot the inverse x
//              transform of the fluctuations u, v, w, p, the in-plane
//              products q = u_i u_i and u_i u_j, their forward transform; the
//              operand blocks X[f][m_x][s][p] and the one-point sums.
//              k1_onepoint: eps (Parseval in x, stencils in y and z) and the
//              one-point parts of the terms.
//   correlate  k1_correlate, one CTA per (tile pair, m_x): the snapshot sums
//              of the correlation products of Eq. 7 (Parseval, Eq. 8-9), 20
//              contractions, each added into the per-pair term spectra with
//              its coefficients; then the one-point parts and the mean-flow
//              couplings.  Only term spectra reach HBM.  A remainder of at
//              most 8 points past the last full tile runs as strips
//              (k1_correlate_strip) instead of as padded tiles.
//   terms      k1_transform_r (nx = 128, 256, 512; register FFT) or
//              k1_transform: the inverse x transform of every (term, pair).
//   stencil    k1_stencil_a: the Step-3 parts -2 nu dA/dr_y, -2 nu dA/dr_z,
//              -(nu/2) dA/dY, -(nu/2) dA/dZ (Eq. 10-11 in y and in z);
//              k1_stencil_res: the residual's r_y, r_z, Y, Z divergences.
//   FP32 plans: operands, contractions, spectra, transforms and stencils
//              in FP32 (means, products pass and one-point sums in FP64);
//              the spectra, transforms and stencils carry the correlation
//              parts only; k1_offsets then adds each pair's rx-independent
//              one-point parts (and their stencil parts), formed in
//              FP64, so that FP32 storage does not round them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/gke1h.h"
#include "gke_common.cuh"

using gke::zd;
using gke::zf;
using gke::mk;
using gke::cplx;

namespace gke1h {

template <typename T> __device__ __forceinline__ cplx<T> cvt(const zd v) { return mk((T)v.x, (T)v.y); }
template <typename T> __device__ __forceinline__ zd wide(const cplx<T> v) { return mk((double)v.x, (double)v.y); }

// operand fields: the fluctuations and the in-plane products
enum Fld { G_U = 0, G_V, G_W, G_P, G_Q, G_UU, G_UV, G_UW, G_VV, G_VW, G_WW, NFLD };
// per-pair term accumulators (the residual is formed at the end)
enum Acc { A_A = 0, A_PHIX, A_PHIY, A_PHIZ, A_PSIY, A_PSIZ, A_XI, NACC };
// one-point sums per point: <u_i u_j> (uu vv ww uv uw vw), <q u_k>, <p v>, <p w>
enum M1 { M_UU = 0, M_VV, M_WW, M_UV, M_UW, M_VW, M_QU, M_QV, M_QW, M_PV, M_PW, NM1 };
// one-point parts of the terms per point: K = <u_i u_i>, <q u_k>, <p u_k>, 2 (Pi - eps)
// (FP32 variant: also the stencil sums of K and of the weights, k1_kgrad)
enum OP { O_K = 0, O_SX, O_SY, O_SZ, O_PY, O_PZ, O_E0, O_DYK, O_DZK, O_SWY, O_SWZ, NOP };
// profile rows (GKE1H_PROF_*)
enum Pr { R_U = 0, R_V, R_W, R_P, R_G, R_EPS = R_G + 6, NPR };

__host__ __device__ inline int prod_field(int i, int k)
{
    const int a = i < k ? i : k, b = i < k ? k : i;
    return a == 0 ? (b == 0 ? G_UU : b == 1 ? G_UV : G_UW) : a == 1 ? (b == 1 ? G_VV : G_VW) : G_WW;
}

// A contraction: sum over its terms t of w_t conj(X[fa_t](p1)) X[fb_t](p2),
// summed over snapshots; added to the accumulators with the constant
// coefficients c[A .. psi_z]; ra >= 0 marks <u_ra(p1) u_rb(p2)'>, whose
// coefficient in xi depends on the pair (k1_correlate).
struct Job { int nt; int fa[8]; int fb[8]; double w[8]; double c[6]; int ra, rb; };
constexpr int NJ = 20;
__constant__ Job c_job[NJ];

static void make_jobs(std::vector<Job>& js)
{
    js.clear();
    auto job = [](std::initializer_list<std::tuple<int, int, double>> terms, std::initializer_list<double> c,
                  int ra = -1, int rb = -1) {
        Job j{};
        j.nt = 0;
        for (auto& t : terms) {
            j.fa[j.nt] = std::get<0>(t); j.fb[j.nt] = std::get<1>(t); j.w[j.nt] = std::get<2>(t); ++j.nt;
        }
        int i = 0;
        for (double v : c) j.c[i++] = v;
        j.ra = ra; j.rb = rb;
        return j;
    };
    // <u_a(p1) u_b(p2)'>: -2 into A when a = b; xi through the mean gradients
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) js.push_back(job({{a, b, 1.0}}, {a == b ? -2.0 : 0.0, 0, 0, 0, 0, 0}, a, b));
    // Phi_x: <du^2 du> = G1 - G2, G1 = <q u'> + 2 <(u_i u) u_i'>, G2 = <u q'> + 2 <u_i (u_i u)'>
    js.push_back(job({{G_Q, G_U, 1.0}, {G_UU, G_U, 2.0}, {G_UV, G_V, 2.0}, {G_UW, G_W, 2.0},
                      {G_U, G_Q, -1.0}, {G_U, G_UU, -2.0}, {G_V, G_UV, -2.0}, {G_W, G_UW, -2.0}},
                     {0, 1.0, 0, 0, 0, 0}));
    for (int k = 1; k <= 2; ++k) {
        const int phi = k == 1 ? 2 : 3, psi = k == 1 ? 4 : 5;
        auto cc = [&](double cphi, double cpsi) {
            std::vector<double> c(6, 0.0);
            c[phi] = cphi; c[psi] = cpsi;
            return c;
        };
        auto jobv = [&](std::vector<std::tuple<int, int, double>> terms, std::vector<double> c) {
            Job j{};
            j.nt = (int)terms.size();
            for (int t = 0; t < j.nt; ++t) {
                j.fa[t] = std::get<0>(terms[t]); j.fb[t] = std::get<1>(terms[t]); j.w[t] = std::get<2>(terms[t]);
            }
            for (int i = 0; i < 6; ++i) j.c[i] = c[i];
            j.ra = j.rb = -1;
            return j;
        };
        // Q1 = <q u_k'>, Q2 = <u_k q'>, X1 = sum_i <(u_i u_k) u_i'>, X2 = sum_i <u_i (u_i u_k)'>:
        // <du^2 du_k> = Q1 + 2 X1 - Q2 - 2 X2, <u_k* du^2> = (Q1 + Q2)/2 - X1 - X2
        js.push_back(jobv({{G_Q, k, 1.0}}, cc(1.0, 0.5)));
        js.push_back(jobv({{k, G_Q, 1.0}}, cc(-1.0, 0.5)));
        js.push_back(jobv({{prod_field(0, k), 0, 1.0}, {prod_field(1, k), 1, 1.0}, {prod_field(2, k), 2, 1.0}},
                          cc(2.0, -1.0)));
        js.push_back(jobv({{0, prod_field(0, k), 1.0}, {1, prod_field(1, k), 1.0}, {2, prod_field(2, k), 1.0}},
                          cc(-2.0, -1.0)));
        // <dp du_k> = <p u_k>(p1) + <p u_k>(p2) - <p u_k'> - <u_k p'>
        js.push_back(jobv({{G_P, k, 1.0}, {k, G_P, 1.0}}, cc(0.0, -2.0)));
    }
}

__host__ __device__ inline long long tri(long long a, long long b, long long P)
{
    return a * P - a * (a - 1) / 2 + (b - a);
}

// ------------------------------------------------------------------- mean
__global__ void k1_mean(const zd* __restrict__ f, int ns, int P, int nxh, double* __restrict__ prof)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    for (int c = 0; c < 4; ++c) {
        double s = 0.0;
        for (int t = 0; t < ns; ++t) s += f[((long long)(t * 4 + c) * P + p) * nxh].x;
        prof[(long long)(R_U + c) * P + p] = s / ns;
    }
}

// d_y U_i, d_z U_i at every point (stencils of the y and z grids)
// (pf != nullptr: also a float copy of the mean and gradient rows, which the
// FP32 correlator's epilogue reads)
__global__ void k1_grad(int ny, int nz, const double* __restrict__ wy, const int* __restrict__ ly,
                        const double* __restrict__ wz, const int* __restrict__ lz, double* __restrict__ prof,
                        float* __restrict__ pf)
{
    const int P = ny * nz;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int iy = p / nz, iz = p - iy * nz;
    for (int i = 0; i < 3; ++i) {
        const double* U = prof + (long long)(R_U + i) * P;
        double gy = 0.0, gz = 0.0;
        for (int l = 0; l < 5; ++l) {
            gy = fma(wy[5 * iy + l], U[(ly[iy] + l) * nz + iz], gy);
            gz = fma(wz[5 * iz + l], U[iy * nz + lz[iz] + l], gz);
        }
        prof[(long long)(R_G + 2 * i) * P + p] = gy;
        prof[(long long)(R_G + 2 * i + 1) * P + p] = gz;
    }
    if (pf)
        for (int r = 0; r < R_EPS; ++r) pf[(long long)r * P + p] = (float)prof[(long long)r * P + p];
}

// --------------------------------------------------------------- products
// One CTA per point p.  Shared memory: two buffers of NFLD - 4 = 7
// sequences of nx complex values and the nx twiddles.  Thread t owns the
// physical points x = t, t + blockDim, ... (at most two: nx <= 512).
// FP64 arithmetic; the operand blocks are stored in TF (double or float).
template <typename TF>
__global__ void __launch_bounds__(256)
k1_products(const zd* __restrict__ f, int ns, int P, int nx, const zd* __restrict__ tw,
            const double* __restrict__ prof, cplx<TF>* __restrict__ X, double* __restrict__ m1, int* __restrict__ bad)
{
    extern __shared__ zd sm[];
    const int nxh = nx / 2 + 1;
    zd* b0 = sm;
    zd* b1 = sm + 7 * nx;
    zd* stw = sm + 14 * nx;
    gke::load_twiddles(stw, tw, nx);
    const int p = blockIdx.x;
    double mean[4];
    for (int c = 0; c < 4; ++c) mean[c] = prof[(long long)(R_U + c) * P + p];
    double acc[NM1];
    for (int k = 0; k < NM1; ++k) acc[k] = 0.0;
    const double inv_nx = 1.0 / nx;
    bool nonfinite = false;
    for (int s = 0; s < ns; ++s) {
        __syncthreads();
        // load the four fields (fluctuations), write their operand blocks,
        // extend to the full Hermitian spectrum
        for (int e = threadIdx.x; e < 4 * nxh; e += blockDim.x) {
            const int c = e / nxh, m = e - c * nxh;
            zd v = f[((long long)(s * 4 + c) * P + p) * nxh + m];
            if (!isfinite(v.x) || !isfinite(v.y)) nonfinite = true;
            if (m == 0) { v.x -= mean[c]; v.y = 0.0; }
            if (2 * m == nx) v.y = 0.0;
            X[(((long long)c * nxh + m) * ns + s) * P + p] = cvt<TF>(v);
            b0[c * nx + m] = v;
            if (m > 0 && 2 * m < nx) b0[c * nx + nx - m] = mk(v.x, -v.y);
        }
        zd* r = gke::fft_block<double, true>(b0, b1, nx, 4, nx, stw);
        zd* o = (r == b0) ? b1 : b0;
        // products on the grid and one-point sums
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const double u = r[x].x, v = r[nx + x].x, w = r[2 * nx + x].x, pp = r[3 * nx + x].x;
            const double uu = u * u, vv = v * v, ww = w * w, uv = u * v, uw = u * w, vw = v * w;
            const double q = uu + vv + ww;
            o[0 * nx + x] = mk(q, 0.0);
            o[1 * nx + x] = mk(uu, 0.0);
            o[2 * nx + x] = mk(uv, 0.0);
            o[3 * nx + x] = mk(uw, 0.0);
            o[4 * nx + x] = mk(vv, 0.0);
            o[5 * nx + x] = mk(vw, 0.0);
            o[6 * nx + x] = mk(ww, 0.0);
            acc[M_UU] += uu; acc[M_VV] += vv; acc[M_WW] += ww;
            acc[M_UV] += uv; acc[M_UW] += uw; acc[M_VW] += vw;
            acc[M_QU] += q * u; acc[M_QV] += q * v; acc[M_QW] += q * w;
            acc[M_PV] += pp * v; acc[M_PW] += pp * w;
        }
        zd* g = gke::fft_block<double, false>(o, r, nx, 7, nx, stw);
        for (int e = threadIdx.x; e < 7 * nxh; e += blockDim.x) {
            const int j = e / nxh, m = e - j * nxh;
            const zd v = g[j * nx + m];
            X[(((long long)(G_Q + j) * nxh + m) * ns + s) * P + p] = cvt<TF>(mk(v.x * inv_nx, v.y * inv_nx));
        }
    }
    // block sums of the one-point statistics
    __shared__ double red[NM1][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < NM1; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < NM1) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        m1[(long long)threadIdx.x * P + p] = v / ((double)ns * nx);
    }
    if (nonfinite) atomicExch(bad, 1);
}

// eps by Parseval in x (signed wavenumber, 0 at the Nyquist index; weight 2
// on the interior wavenumbers) with stencil derivatives in y and z of the
// operand blocks; then the one-point parts of the terms.  One CTA per point:
// the threads share the (component, wavenumber, snapshot) triples.
template <typename TF>
__global__ void __launch_bounds__(128)
k1_onepoint(const cplx<TF>* __restrict__ X, int ns, int ny, int nz, int nx, double kx0, double nu,
            const double* __restrict__ wy, const int* __restrict__ ly, const double* __restrict__ wz,
            const int* __restrict__ lz, const double* __restrict__ m1, double* __restrict__ prof,
            double* __restrict__ op)
{
    const int P = ny * nz, nxh = nx / 2 + 1;
    const int p = blockIdx.x;
    const int iy = p / nz, iz = p - iy * nz;
    double e = 0.0;
    for (int t = threadIdx.x; t < 3 * nxh * ns; t += blockDim.x) {
        const int i = t / (nxh * ns), r = t - i * nxh * ns, m = r / ns, s = r - m * ns;
        const double k = (2 * m == nx) ? 0.0 : kx0 * m;
        const double ck = (m == 0 || 2 * m == nx) ? 1.0 : 2.0;
        const cplx<TF>* row = X + (((long long)i * nxh + m) * ns + s) * P;
        const zd a = wide(row[p]);
        zd dy = mk(0.0, 0.0), dz = mk(0.0, 0.0);
        for (int l = 0; l < 5; ++l) {
            const zd t1 = wide(row[(ly[iy] + l) * nz + iz]), t2 = wide(row[iy * nz + lz[iz] + l]);
            dy.x = fma(wy[5 * iy + l], t1.x, dy.x); dy.y = fma(wy[5 * iy + l], t1.y, dy.y);
            dz.x = fma(wz[5 * iz + l], t2.x, dz.x); dz.y = fma(wz[5 * iz + l], t2.y, dz.y);
        }
        e += ck * (k * k * (a.x * a.x + a.y * a.y) + dy.x * dy.x + dy.y * dy.y + dz.x * dz.x + dz.y * dz.y);
    }
    __shared__ double red[4];
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x != 0) return;
    e = red[0] + red[1] + red[2] + red[3];
    const double eps = nu * e / ns;
    prof[(long long)R_EPS * P + p] = eps;
    auto M = [&](int k) { return m1[(long long)k * P + p]; };
    auto G = [&](int i, int k) { return prof[(long long)(R_G + 2 * i + k - 1) * P + p]; };
    // production -<u_i u_k> d_k U_i over i = x, y, z and k = y, z
    const double Pi = -(M(M_UV) * G(0, 1) + M(M_VV) * G(1, 1) + M(M_VW) * G(2, 1) +
                        M(M_UW) * G(0, 2) + M(M_VW) * G(1, 2) + M(M_WW) * G(2, 2));
    op[(long long)O_K * P + p] = M(M_UU) + M(M_VV) + M(M_WW);
    op[(long long)O_SX * P + p] = M(M_QU);
    op[(long long)O_SY * P + p] = M(M_QV);
    op[(long long)O_SZ * P + p] = M(M_QW);
    op[(long long)O_PY * P + p] = M(M_PV);
    op[(long long)O_PZ * P + p] = M(M_PW);
    op[(long long)O_E0 * P + p] = 2.0 * (Pi - eps);
}

// FP32 variant: per point, the stencil sums of K = <u_i u_i> and of the
// weights in y and z (the offsets' stencil parts, k1_offsets)
__global__ void k1_kgrad(int ny, int nz, const double* __restrict__ wy, const int* __restrict__ ly,
                         const double* __restrict__ wz, const int* __restrict__ lz, double* __restrict__ op)
{
    const int P = ny * nz;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int iy = p / nz, iz = p - iy * nz;
    const double* K = op + (long long)O_K * P;
    double dy = 0.0, dz = 0.0, sy = 0.0, sz = 0.0;
    for (int l = 0; l < 5; ++l) {
        dy = fma(wy[5 * iy + l], K[(ly[iy] + l) * nz + iz], dy);
        dz = fma(wz[5 * iz + l], K[iy * nz + lz[iz] + l], dz);
        sy += wy[5 * iy + l];
        sz += wz[5 * iz + l];
    }
    op[(long long)O_DYK * P + p] = dy;
    op[(long long)O_DZK * P + p] = dz;
    op[(long long)O_SWY * P + p] = sy;
    op[(long long)O_SWZ * P + p] = sz;
}

// -------------------------------------------------------------- correlate
#define CT 32        // tile edge (points)
#define SCH 8        // snapshots per shared-memory chunk
#define STRIP_MAX 8  // widest remainder past the last full tile done as strips

template <typename T>
__device__ __forceinline__ void cmac(cplx<T>& acc, const cplx<T> a, const cplx<T> b)     // acc += conj(a) b
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

// add contraction jb's value at (q1, q2) into the accumulators of that pair
template <typename TA>
__device__ __forceinline__ void add_job(cplx<TA>* T, const Job& jb, const cplx<TA> acc, int q1, int q2, int P,
                                        const TA* __restrict__ prof)
{
    #pragma unroll
    for (int t = 0; t < 6; ++t) {
        const TA c = (TA)jb.c[t];
        if (c == (TA)0) continue;
        T[t].x = fma(c, acc.x, T[t].x);
        T[t].y = fma(c, acc.y, T[t].y);
    }
    if (jb.ra >= 0) {
        // xi: <u_a(p1) u_b(p2)'> enters -2 <du_i du_k> (d_k U_i)* - 2 <du_i u_k*> d(d_k U_i)
        // with weight 2 d_b U_a(p2) (b = y, z) + 2 d_a U_b(p1) (a = y, z)
        const int ra = jb.ra, rb = jb.rb;
        TA c = (TA)0;
        if (rb >= 1 && q2 < P) c += (TA)2 * prof[(long long)(R_G + 2 * ra + rb - 1) * P + q2];
        if (ra >= 1 && q1 < P) c += (TA)2 * prof[(long long)(R_G + 2 * rb + ra - 1) * P + q1];
        T[A_XI].x = fma(c, acc.x, T[A_XI].x);
        T[A_XI].y = fma(c, acc.y, T[A_XI].y);
    }
}

// snapshot average, one-point parts (m = 0), mean-flow couplings and the
// residual's spectral part; writes the eight spectra of pair (q1 <= q2).
// Arithmetic in TF; pt holds the mean and gradient rows in TF.
template <typename TF>
__device__ __forceinline__ void finish_pair(const cplx<TF>* T, int q1, int q2, int m, int nx, double kx0, double nu_,
                                            int ns, int P, const TF* __restrict__ pt,
                                            const double* __restrict__ op, cplx<TF>* __restrict__ spec,
                                            long long npair)
{
    typedef cplx<TF> C;
    const int nxh = nx / 2 + 1;
    const TF inv = (TF)1 / (TF)ns, nu = (TF)nu_;
    const TF k = (2 * m == nx) ? (TF)0 : (TF)(kx0 * m);
    C v[NACC];
    #pragma unroll
    for (int t = 0; t < NACC; ++t) v[t] = mk(T[t].x * inv, T[t].y * inv);
    auto O = [&](int r, int q) { return op[(long long)r * P + q]; };
    auto U = [&](int r, int q) { return pt[(long long)r * P + q]; };
    // FP64 spectra carry the one-point parts at m = 0; FP32 spectra leave them
    // (and their mean-flow couplings) to k1_offsets, which adds them in FP64
    // after the stencils, so that FP32 storage does not round them
    if (m == 0 && sizeof(TF) == 8) {
        v[A_A].x += O(O_K, q1) + O(O_K, q2);
        v[A_PHIX].x += O(O_SX, q2) - O(O_SX, q1);
        v[A_PHIY].x += O(O_SY, q2) - O(O_SY, q1);
        v[A_PHIZ].x += O(O_SZ, q2) - O(O_SZ, q1);
        v[A_PSIY].x += 0.5 * (O(O_SY, q1) + O(O_SY, q2)) + 2.0 * (O(O_PY, q1) + O(O_PY, q2));
        v[A_PSIZ].x += 0.5 * (O(O_SZ, q1) + O(O_SZ, q2)) + 2.0 * (O(O_PZ, q1) + O(O_PZ, q2));
        v[A_XI].x += O(O_E0, q1) + O(O_E0, q2);
    }
    const C A = v[A_A];
    const TF dU = U(R_U, q2) - U(R_U, q1), dV = U(R_V, q2) - U(R_V, q1), dW = U(R_W, q2) - U(R_W, q1);
    const TF h = (TF)0.5, two = (TF)2;
    const TF Vs = h * (U(R_V, q1) + U(R_V, q2)), Ws = h * (U(R_W, q1) + U(R_W, q2));
    // Phi_x += dU A - 2 nu (i k) A
    v[A_PHIX].x += dU * A.x + two * nu * k * A.y;
    v[A_PHIX].y += dU * A.y - two * nu * k * A.x;
    v[A_PHIY].x += dV * A.x; v[A_PHIY].y += dV * A.y;
    v[A_PHIZ].x += dW * A.x; v[A_PHIZ].y += dW * A.y;
    v[A_PSIY].x += Vs * A.x; v[A_PSIY].y += Vs * A.y;
    v[A_PSIZ].x += Ws * A.x; v[A_PSIZ].y += Ws * A.y;
    // residual spectrum: i k Phi_x - xi (the stencil parts come later)
    const C res = mk(-k * v[A_PHIX].y - v[A_XI].x, k * v[A_PHIX].x - v[A_XI].y);
    const long long pr = tri(q1, q2, P);
    #pragma unroll
    for (int t = 0; t < NACC; ++t) spec[((long long)t * nxh + m) * npair + pr] = v[t];
    spec[((long long)NACC * nxh + m) * npair + pr] = res;
}

// CTA = (tile pair T1 <= T2 of the nt full tiles, wavenumber m); 16 x 16
// threads, each an RB x RB block of pairs (p1 = T1 CT + ty + 16 a,
// p2 = T2 CT + tx + 16 b).  With strips, the points past the last full tile
// are left to k1_correlate_strip; otherwise the last tile is padded.
template <typename TF>
__global__ void __launch_bounds__(256, sizeof(TF) == 4 ? 2 : 1)
k1_correlate(const cplx<TF>* __restrict__ X, int ns, int P, int nx, int nt, double kx0, double nu,
             const TF* __restrict__ prof, const double* __restrict__ op, cplx<TF>* __restrict__ spec,
             long long npair)
{
    typedef cplx<TF> C;
    constexpr int RB = 2;
    constexpr int SC = sizeof(TF) == 4 ? 2 * SCH : SCH;     // snapshots per staged chunk
    __shared__ C As[SC][CT];
    __shared__ C Bs[SC][CT];
    const int nxh = nx / 2 + 1;
    const int m = blockIdx.y;
    int T1 = 0, rem = blockIdx.x;
    while (rem >= nt - T1) { rem -= nt - T1; ++T1; }
    const int T2 = T1 + rem;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int p1[RB], p2[RB];
    for (int a = 0; a < RB; ++a) { p1[a] = T1 * CT + ty + 16 * a; p2[a] = T2 * CT + tx + 16 * a; }
    C T[NACC][RB][RB];
    #pragma unroll
    for (int t = 0; t < NACC; ++t)
        #pragma unroll
        for (int a = 0; a < RB; ++a)
            #pragma unroll
            for (int b = 0; b < RB; ++b) T[t][a][b] = mk((TF)0, (TF)0);
    for (int j = 0; j < NJ; ++j) {
        const Job& jb = c_job[j];
        C acc[RB][RB];
        #pragma unroll
        for (int a = 0; a < RB; ++a)
            #pragma unroll
            for (int b = 0; b < RB; ++b) acc[a][b] = mk((TF)0, (TF)0);
        for (int t = 0; t < jb.nt; ++t) {
            // the term's weight (real) scales its A operand as it is staged:
            // conj(w a) b = w conj(a) b, so the sum goes straight into acc
            const TF wt = (TF)jb.w[t];
            const C* A = X + ((long long)jb.fa[t] * nxh + m) * ns * P;
            const C* B = X + ((long long)jb.fb[t] * nxh + m) * ns * P;
            for (int s0 = 0; s0 < ns; s0 += SC) {
                __syncthreads();
                for (int e = threadIdx.x; e < SC * CT; e += blockDim.x) {
                    const int ss = e / CT, yy = e - ss * CT, s = s0 + ss;
                    C va = mk((TF)0, (TF)0), vb = va;
                    if (s < ns && T1 * CT + yy < P) { va = A[(long long)s * P + T1 * CT + yy]; va.x *= wt; va.y *= wt; }
                    if (s < ns && T2 * CT + yy < P) vb = B[(long long)s * P + T2 * CT + yy];
                    As[ss][yy] = va;
                    Bs[ss][yy] = vb;
                }
                __syncthreads();
                #pragma unroll
                for (int ss = 0; ss < SC; ++ss) {
                    C av[RB], bv[RB];
                    #pragma unroll
                    for (int i = 0; i < RB; ++i) { av[i] = As[ss][ty + 16 * i]; bv[i] = Bs[ss][tx + 16 * i]; }
                    #pragma unroll
                    for (int a = 0; a < RB; ++a)
                        #pragma unroll
                        for (int b = 0; b < RB; ++b) cmac(acc[a][b], av[a], bv[b]);
                }
            }
        }
        // the contraction into the term spectra (as add_job, one coefficient test per job)
        #pragma unroll
        for (int t = 0; t < 6; ++t) {
            const TF c = (TF)jb.c[t];
            if (c == (TF)0) continue;
            #pragma unroll
            for (int a = 0; a < RB; ++a)
                #pragma unroll
                for (int b = 0; b < RB; ++b) {
                    T[t][a][b].x = fma(c, acc[a][b].x, T[t][a][b].x);
                    T[t][a][b].y = fma(c, acc[a][b].y, T[t][a][b].y);
                }
        }
        if (jb.ra >= 0) {
            const int ra = jb.ra, rb = jb.rb;
            #pragma unroll
            for (int a = 0; a < RB; ++a)
                #pragma unroll
                for (int b = 0; b < RB; ++b) {
                    TF c = (TF)0;
                    if (rb >= 1 && p2[b] < P) c += (TF)2 * prof[(long long)(R_G + 2 * ra + rb - 1) * P + p2[b]];
                    if (ra >= 1 && p1[a] < P) c += (TF)2 * prof[(long long)(R_G + 2 * rb + ra - 1) * P + p1[a]];
                    T[A_XI][a][b].x = fma(c, acc[a][b].x, T[A_XI][a][b].x);
                    T[A_XI][a][b].y = fma(c, acc[a][b].y, T[A_XI][a][b].y);
                }
        }
    }
    #pragma unroll
    for (int a = 0; a < RB; ++a)
        #pragma unroll
        for (int b = 0; b < RB; ++b) {
            if (p1[a] >= P || p2[b] >= P || p2[b] < p1[a]) continue;
            C v[NACC];
            #pragma unroll
            for (int t = 0; t < NACC; ++t) v[t] = T[t][a][b];
            finish_pair<TF>(v, p1[a], p2[b], m, nx, kx0, nu, ns, P, prof, op, spec, npair);
        }
}

// The pairs (p1 <= p2) with p2 >= cov (the points past the last full tile):
// one thread per (pair, wavenumber), the same contractions one pair at a time;
// consecutive threads take consecutive p1 (coalesced operand loads).
template <typename TF>
__global__ void __launch_bounds__(128)
k1_correlate_strip(const cplx<TF>* __restrict__ X, int ns, int P, int nx, int cov, double kx0, double nu,
                   const TF* __restrict__ prof, const double* __restrict__ op, cplx<TF>* __restrict__ spec,
                   long long npair)
{
    typedef cplx<TF> C;
    const int nxh = nx / 2 + 1;
    const int rem = P - cov;
    // pairs of the strip: p2 = cov + r, p1 = 0 .. p2; n = rem cov + rem (rem + 1) / 2
    const long long n = (long long)rem * cov + (long long)rem * (rem + 1) / 2;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nxh) return;
    const int m = (int)(e / n);                       // consecutive threads: consecutive p1 of one p2
    long long k = e - (long long)m * n;
    int r = 0;
    while (k >= cov + r + 1) { k -= cov + r + 1; ++r; }
    const int q2 = cov + r, q1 = (int)k;
    C T[NACC];
    #pragma unroll
    for (int t = 0; t < NACC; ++t) T[t] = mk((TF)0, (TF)0);
    for (int j = 0; j < NJ; ++j) {
        const Job& jb = c_job[j];
        C acc = mk((TF)0, (TF)0);
        for (int t = 0; t < jb.nt; ++t) {
            const C* A = X + ((long long)jb.fa[t] * nxh + m) * ns * P;
            const C* B = X + ((long long)jb.fb[t] * nxh + m) * ns * P;
            C part = mk((TF)0, (TF)0);
            for (int s = 0; s < ns; ++s) cmac(part, A[(long long)s * P + q1], B[(long long)s * P + q2]);
            acc.x = fma((TF)jb.w[t], part.x, acc.x);
            acc.y = fma((TF)jb.w[t], part.y, acc.y);
        }
        add_job(T, jb, acc, q1, q2, P, prof);
    }
    finish_pair<TF>(T, q1, q2, m, nx, kx0, nu, ns, P, prof, op, spec, npair);
}

// ------------------------------------------------------------- transforms
// CTA = 2 NB consecutive pairs of one term.  The spectra (nx/2 + 1
// wavenumbers each, imaginary parts dropped at m = 0 and m = nx/2) are
// staged in shared memory; pairs 2b and 2b + 1 share one complex sequence,
// H_2b + i H_2b+1 with H the Hermitian extension, whose inverse transform
// has the two real correlations as its real and imaginary parts.
template <typename TF>
__global__ void __launch_bounds__(256)
k1_transform(const cplx<TF>* __restrict__ spec, int nx, long long npair, int NB, const cplx<TF>* __restrict__ tw,
             TF* __restrict__ terms)
{
    typedef cplx<TF> C;
    extern __shared__ __align__(16) unsigned char sm_tr[];
    C* sm = (C*)sm_tr;
    const int nxh = nx / 2 + 1;
    C* b0 = sm;
    C* b1 = sm + (size_t)NB * nx;
    C* stw = sm + (size_t)2 * NB * nx;
    C* stg = stw + nx;                                // [2 NB][nxh]
    gke::load_twiddles(stw, tw, nx);
    const int t = blockIdx.y;
    const long long pr0 = (long long)blockIdx.x * 2 * NB;
    const int np = (int)std::min<long long>(2 * NB, npair - pr0);
    for (int e = threadIdx.x; e < nxh * 2 * NB; e += blockDim.x) {
        const int m = e / (2 * NB), c = e - m * 2 * NB;
        C v = mk((TF)0, (TF)0);
        if (c < np) v = spec[((long long)t * nxh + m) * npair + pr0 + c];
        if (m == 0 || 2 * m == nx) v.y = (TF)0;
        stg[c * nxh + m] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NB * nx; e += blockDim.x) {
        const int b = e / nx, k = e - b * nx;
        const bool lo = 2 * k <= nx;
        const C a = stg[(2 * b) * nxh + (lo ? k : nx - k)];
        const C c = stg[(2 * b + 1) * nxh + (lo ? k : nx - k)];
        const TF ay = lo ? a.y : -a.y, cy = lo ? c.y : -c.y;
        b0[b * nx + k] = mk(a.x - cy, ay + c.x);
    }
    C* r = gke::fft_block<TF, true>(b0, b1, nx, NB, nx, stw);
    for (int e = threadIdx.x; e < np * nx; e += blockDim.x) {
        const int c = e / nx, x = e - c * nx;
        const C z = r[(c >> 1) * nx + x];
        terms[((long long)t * npair + pr0 + c) * nx + x] = (c & 1) ? z.y : z.x;
    }
}

// Register-FFT variant for nx = N1 N2 (gke::fft2l, twiddles resolved at
// compile time): CTA = RZ sequences x N2 lanes, each sequence two pairs
// packed as above; lane l holds the wavenumbers l + N2 j of its sequence.
template <typename TF, int N1, int N2>
__global__ void __launch_bounds__(256)
k1_transform_r(const cplx<TF>* __restrict__ spec, long long npair, const cplx<TF>* __restrict__ tw,
               TF* __restrict__ terms)
{
    typedef cplx<TF> C;
    constexpr int N = N1 * N2, nxh = N / 2 + 1, RZ = 256 / N2;
    extern __shared__ __align__(16) unsigned char sm_trr[];
    C* stw = (C*)sm_trr;
    C* xs = stw + N;
    const int lane = threadIdx.x % N2, r = threadIdx.x / N2;
    const int t = blockIdx.y;
    const long long pa = ((long long)blockIdx.x * RZ + r) * 2, pb = pa + 1;
    const bool la = pa < npair, lb = pb < npair;
    gke::load_twiddles(stw, tw, N);
    // spectra [t][m][pair]: the two pairs of a sequence share 32-byte sectors
    const C* sa = spec + (long long)t * nxh * npair + (la ? pa : 0);
    const C* sb = spec + (long long)t * nxh * npair + (lb ? pb : 0);
    C v[N1];
    #pragma unroll
    for (int j = 0; j < N1; ++j) {
        const int k = lane + N2 * j;
        const bool lo = 2 * k <= N;
        C a = mk((TF)0, (TF)0), b = a;
        if (la) { a = sa[(long long)(lo ? k : N - k) * npair]; if (!lo) a.y = -a.y; }
        if (lb) { b = sb[(long long)(lo ? k : N - k) * npair]; if (!lo) b.y = -b.y; }
        if (k == 0 || 2 * k == N) { a.y = (TF)0; b.y = (TF)0; }
        v[j] = mk(a.x - b.y, a.y + b.x);
    }
    __syncthreads();                                  // twiddles staged
    gke::fft2l<TF, N1, N2, true>(v, lane, xs + r * N1 * (N2 + 1), N2 + 1, 1, stw);
    #pragma unroll
    for (int j = 0; j < N1; ++j) {
        const int x = lane + N2 * j;
        if (la) terms[((long long)t * npair + pa) * N + x] = v[j].x;
        if (lb) terms[((long long)t * npair + pb) * N + x] = v[j].y;
    }
}

// --------------------------------------------------------------- stencils
// CTA = G pairs (4, or 256 / nx below nx = 64).  The 20 neighbour pairs of each pair
// (5 stencil nodes in each of Y1, Y2, Z1, Z2) are resolved once per CTA into
// shared memory: the offset of the stored pair's row and whether it is the
// r-inverted one (q1 > q2: read (q2, q1) at -m, times the term's parity).
struct Sten { const double* wy; const int* ly; const double* wz; const int* lz; int ny, nz; };

constexpr int SG = 32;        // most pairs per CTA (nx >= 8)

template <typename TW>
__device__ __forceinline__ void neighbours(const Sten& S, const int* __restrict__ pq, long long pr0, int G,
                                           int nx, long long npair, long long (*off)[20], signed char (*flip)[20],
                                           TW (*w)[20])
{
    const int P = S.ny * S.nz;
    for (int e = threadIdx.x; e < G * 20; e += blockDim.x) {
        const int g = e / 20, j = e - g * 20, dir = j / 5, l = j - dir * 5;
        const long long pr = pr0 + g;
        if (pr >= npair) continue;
        const int q1 = pq[2 * pr], q2 = pq[2 * pr + 1];
        const int iy1 = q1 / S.nz, iz1 = q1 - iy1 * S.nz, iy2 = q2 / S.nz, iz2 = q2 - iy2 * S.nz;
        int a = q1, b = q2;
        double wt;
        if (dir == 0)      { a = (S.ly[iy1] + l) * S.nz + iz1; wt = S.wy[5 * iy1 + l]; }
        else if (dir == 1) { b = (S.ly[iy2] + l) * S.nz + iz2; wt = S.wy[5 * iy2 + l]; }
        else if (dir == 2) { a = iy1 * S.nz + S.lz[iz1] + l;   wt = S.wz[5 * iz1 + l]; }
        else               { b = iy2 * S.nz + S.lz[iz2] + l;   wt = S.wz[5 * iz2 + l]; }
        const bool f = a > b;
        off[g][j] = tri(f ? b : a, f ? a : b, P) * nx;
        flip[g][j] = f ? 1 : 0;
        w[g][j] = (TW)wt;                               // converted once, not per use
    }
    __syncthreads();
}

// d_Y1, d_Y2, d_Z1, d_Z2 of one plane at separation m of CTA pair g
// (arithmetic in the terms' type TO)
template <typename TO>
__device__ __forceinline__ void derivs4(const TO* __restrict__ plane, const long long* off,
                                        const signed char* flip, const TO* w, int m, int nx, TO sg, TO d[4])
{
    const int mm = m == 0 ? 0 : nx - m;
    #pragma unroll
    for (int dir = 0; dir < 4; ++dir) {
        TO acc = (TO)0;
        #pragma unroll
        for (int l = 0; l < 5; ++l) {
            const int j = 5 * dir + l;
            const TO v = flip[j] ? sg * plane[off[j] + mm] : plane[off[j] + m];
            acc = fma(w[j], v, acc);
        }
        d[dir] = acc;
    }
}

template <typename TO>
__global__ void __launch_bounds__(256)
k1_stencil_a(TO* __restrict__ terms, const int* __restrict__ pq, Sten S, int nx, long long npair, double nu_)
{
    const TO nu = (TO)nu_;
    __shared__ long long off[SG][20];
    __shared__ signed char flip[SG][20];
    __shared__ TO w[SG][20];
    const int G = nx >= 64 ? 4 : 256 / nx;
    const long long pr0 = (long long)blockIdx.x * G;
    neighbours(S, pq, pr0, G, nx, npair, off, flip, w);
    const TO* Ap = terms + (long long)GKE1H_TERM_A * npair * nx;
    for (int e = threadIdx.x; e < G * nx; e += blockDim.x) {
        const int g = e / nx, m = e - g * nx;
        const long long pr = pr0 + g;
        if (pr >= npair) continue;
        TO d[4];
        derivs4<TO>(Ap, off[g], flip[g], w[g], m, nx, (TO)1, d);
        const TO h = (TO)0.5;
        terms[((long long)GKE1H_TERM_PHI_Y * npair + pr) * nx + m] -= nu * (d[1] - d[0]);
        terms[((long long)GKE1H_TERM_PHI_Z * npair + pr) * nx + m] -= nu * (d[3] - d[2]);
        terms[((long long)GKE1H_TERM_PSI_Y * npair + pr) * nx + m] -= h * nu * (d[0] + d[1]);
        terms[((long long)GKE1H_TERM_PSI_Z * npair + pr) * nx + m] -= h * nu * (d[2] + d[3]);
    }
}

template <typename TO>
__global__ void __launch_bounds__(256)
k1_stencil_res(TO* __restrict__ terms, const int* __restrict__ pq, Sten S, int nx, long long npair)
{
    __shared__ long long off[SG][20];
    __shared__ signed char flip[SG][20];
    __shared__ TO w[SG][20];
    const int G = nx >= 64 ? 4 : 256 / nx;
    const long long pr0 = (long long)blockIdx.x * G;
    neighbours(S, pq, pr0, G, nx, npair, off, flip, w);
    auto plane = [&](int t) { return terms + (long long)t * npair * nx; };
    for (int e = threadIdx.x; e < G * nx; e += blockDim.x) {
        const int g = e / nx, m = e - g * nx;
        const long long pr = pr0 + g;
        if (pr >= npair) continue;
        TO fy[4], fz[4], sy[4], sz[4];
        derivs4<TO>(plane(GKE1H_TERM_PHI_Y), off[g], flip[g], w[g], m, nx, (TO)-1, fy);
        derivs4<TO>(plane(GKE1H_TERM_PHI_Z), off[g], flip[g], w[g], m, nx, (TO)-1, fz);
        derivs4<TO>(plane(GKE1H_TERM_PSI_Y), off[g], flip[g], w[g], m, nx, (TO)1, sy);
        derivs4<TO>(plane(GKE1H_TERM_PSI_Z), off[g], flip[g], w[g], m, nx, (TO)1, sz);
        const TO h = (TO)0.5;
        terms[((long long)GKE1H_TERM_RESIDUAL * npair + pr) * nx + m] +=
            h * (fy[1] - fy[0]) + h * (fz[3] - fz[2]) + (sy[0] + sy[1]) + (sz[2] + sz[3]);
    }
}

// ------------------------------------------------- FP32 variant: offsets
// The rx-independent part of each term of the ordered pair (a, b) (any
// order), from the per-point one-point sums and profiles, in FP64: the
// one-point parts, their mean-flow couplings and the stencil parts of
// A_0 = K(a) + K(b) (Eq. 10-11 in y and z).  o[0..6]: A, Phi_x, Phi_y,
// Phi_z, psi_y, psi_z, xi.
__device__ void pair_offsets(const Sten& S, const double* __restrict__ prof, const double* __restrict__ op,
                             double nu, int a, int b, double o[7])
{
    const int P = S.ny * S.nz;
    auto K = [&](int q) { return op[(long long)O_K * P + q]; };
    auto O = [&](int r, int q) { return op[(long long)r * P + q]; };
    auto U = [&](int r, int q) { return prof[(long long)r * P + q]; };
    // the stencils of A_0 = K(a) + K(b): d_Y1 A_0 = sum_l w_l K(node_l) + K(b) sum_l w_l, etc.
    const double A0 = K(a) + K(b);
    const double y1 = O(O_DYK, a) + K(b) * O(O_SWY, a), y2 = K(a) * O(O_SWY, b) + O(O_DYK, b);
    const double z1 = O(O_DZK, a) + K(b) * O(O_SWZ, a), z2 = K(a) * O(O_SWZ, b) + O(O_DZK, b);
    o[0] = A0;
    o[1] = O(O_SX, b) - O(O_SX, a) + (U(R_U, b) - U(R_U, a)) * A0;
    o[2] = O(O_SY, b) - O(O_SY, a) + (U(R_V, b) - U(R_V, a)) * A0 - nu * (y2 - y1);
    o[3] = O(O_SZ, b) - O(O_SZ, a) + (U(R_W, b) - U(R_W, a)) * A0 - nu * (z2 - z1);
    o[4] = 0.5 * (O(O_SY, a) + O(O_SY, b)) + 2.0 * (O(O_PY, a) + O(O_PY, b)) + 0.5 * (U(R_V, a) + U(R_V, b)) * A0
           - 0.5 * nu * (y1 + y2);
    o[5] = 0.5 * (O(O_SZ, a) + O(O_SZ, b)) + 2.0 * (O(O_PZ, a) + O(O_PZ, b)) + 0.5 * (U(R_W, a) + U(R_W, b)) * A0
           - 0.5 * nu * (z1 + z2);
    o[6] = O(O_E0, a) + O(O_E0, b);
}

// Adds the offsets of every pair to its eight planes; the residual's offset
// is -xi_0 plus the stencil divergences of the offsets of Phi_y, Phi_z,
// psi_y, psi_z over the 20 neighbour pairs.  CTA = G pairs (12, or 256 / nx
// below nx = 64); 21 threads per pair evaluate the pair's and its
// neighbours' offsets.
template <typename TO>
__global__ void __launch_bounds__(256)
k1_offsets(TO* __restrict__ terms, const int* __restrict__ pq, Sten S, int nx, long long npair,
           const double* __restrict__ prof, const double* __restrict__ op, double nu)
{
    __shared__ double so[SG][8];                    // per pair: 7 offsets + the residual's
    __shared__ double sc[SG][21];
    const int G = nx >= 64 ? 12 : 256 / nx;
    const long long pr0 = (long long)blockIdx.x * G;
    for (int e = threadIdx.x; e < G * 21; e += blockDim.x) {
        const int g = e / 21, j = e - g * 21;
        const long long pr = pr0 + g;
        if (pr >= npair) continue;
        const int q1 = pq[2 * pr], q2 = pq[2 * pr + 1];
        double o[7];
        if (j == 20) {
            pair_offsets(S, prof, op, nu, q1, q2, o);
            for (int t = 0; t < 7; ++t) so[g][t] = o[t];
            sc[g][20] = -o[6];
            continue;
        }
        const int dir = j / 5, l = j - dir * 5;
        const int iy1 = q1 / S.nz, iz1 = q1 - iy1 * S.nz, iy2 = q2 / S.nz, iz2 = q2 - iy2 * S.nz;
        int a = q1, b = q2;
        double w;
        if (dir == 0)      { a = (S.ly[iy1] + l) * S.nz + iz1; w = S.wy[5 * iy1 + l]; }
        else if (dir == 1) { b = (S.ly[iy2] + l) * S.nz + iz2; w = S.wy[5 * iy2 + l]; }
        else if (dir == 2) { a = iy1 * S.nz + S.lz[iz1] + l;   w = S.wz[5 * iz1 + l]; }
        else               { b = iy2 * S.nz + S.lz[iz2] + l;   w = S.wz[5 * iz2 + l]; }
        pair_offsets(S, prof, op, nu, a, b, o);
        // d/dr = (d_2 - d_1)/2 on Phi, d/dX = d_1 + d_2 on psi
        const double sgn = (dir & 1) ? 0.5 : -0.5;
        sc[g][j] = dir < 2 ? w * (sgn * o[2] + o[4]) : w * (sgn * o[3] + o[5]);
    }
    __syncthreads();
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        double r = 0.0;
        for (int j = 0; j < 21; ++j) r += sc[g][j];
        so[g][7] = r;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < G * nx; e += blockDim.x) {
        const int g = e / nx, m = e - g * nx;
        const long long pr = pr0 + g;
        if (pr >= npair) continue;
        // added in TO: a conversion to FP64 and back would run on the FP64 pipe
        #pragma unroll
        for (int t = 0; t < GKE1H_NTERM; ++t) {
            TO* v = terms + ((long long)t * npair + pr) * nx + m;
            *v += (TO)so[g][t];
        }
    }
}

}  // namespace gke1h

// =================================================================== plan
using namespace gke1h;

struct gke1h_plan_s {
    int nx = 0, ny = 0, nz = 0, P = 0, nxh = 0, max_snap = 0, nt = 0;
    long long npair = 0;
    double Lx = 0, nu = 0;
    bool f32 = false;                    // GKE_PREC_F32: operands, spectra and terms in FP32
    cudaStream_t st = nullptr;
    double *wy = nullptr, *wz = nullptr, *prof = nullptr, *m1 = nullptr, *op = nullptr;
    int *ly = nullptr, *lz = nullptr, *pq = nullptr, *bad = nullptr;
    zd *tw = nullptr, *fin = nullptr;
    zf* twf = nullptr;
    float* pf = nullptr;                 // float copy of the mean and gradient rows (FP32 plans)
    void *X = nullptr, *spec = nullptr, *terms = nullptr;
    int smem_prod = 0, smem_tr = 0, NB = 0;
    bool reg_tr = false;                 // register-FFT transform (nx = 128, 256, 512)
    bool timing = false;
    struct Mark { int stage; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    long long launches = 0;
    std::string err;
};

static thread_local std::string g1_err;

static gke_status fail1(gke1h_plan_t p, gke_status s, const std::string& m)
{
    if (p) p->err = m; else g1_err = m;
    return s;
}

#define TRY1(p, call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail1(p, e_ == cudaErrorMemoryAllocation ? GKE_ERR_OOM : GKE_ERR_CUDA,    \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                \
    } while (0)

static bool on_device(const void* ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void free_plan(gke1h_plan_t p)
{
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st); else cudaDeviceSynchronize();
    void* bufs[] = {p->wy, p->wz, p->prof, p->m1, p->op, p->terms, p->ly, p->lz, p->pq, p->bad,
                    p->tw, p->twf, p->pf, p->X, p->spec, p->fin};
    for (void* b : bufs) if (b) cudaFree(b);
    for (auto& mk_ : p->marks) { cudaEventDestroy(mk_.a); cudaEventDestroy(mk_.b); }
    delete p;
}

static bool fft_size_ok(int n)
{
    if (n < 8 || n > 512) return false;
    int m = n % 3 == 0 ? n / 3 : n;
    return (m & (m - 1)) == 0;
}

template <typename TF>
static cudaError_t set_attrs(gke1h_plan_t p)
{
    typedef cplx<TF> C;
    cudaError_t e = cudaFuncSetAttribute(k1_products<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, p->smem_prod);
    if (e != cudaSuccess) return e;
    if (p->nx == 128 || p->nx == 256 || p->nx == 512) {
        const void* fn = p->nx == 128 ? (const void*)k1_transform_r<TF, 16, 8>
                       : p->nx == 256 ? (const void*)k1_transform_r<TF, 16, 16>
                                      : (const void*)k1_transform_r<TF, 32, 16>;
        const int n2 = p->nx == 128 ? 8 : 16, n1 = p->nx / n2;
        p->smem_tr = (int)(sizeof(C) * (p->nx + (256 / n2) * n1 * (n2 + 1)));
        p->reg_tr = true;
        return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->smem_tr);
    }
    p->smem_tr = (int)(sizeof(C) * (3 * p->NB * p->nx + 2 * p->NB + p->nx));
    return cudaFuncSetAttribute(k1_transform<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, p->smem_tr);
}

extern "C" gke_status gke1h_plan(const gke1h_desc* d, void* stream, gke1h_plan_t* out)
{
    if (!d || !out) return fail1(nullptr, GKE_ERR_ARG, "NULL descriptor or output");
    *out = nullptr;
    if (d->ny < 5 || d->nz < 5 || !d->y || !d->z || d->max_snap < 1 || !(d->Lx > 0) || !(d->nu > 0))
        return fail1(nullptr, GKE_ERR_ARG, "bad sizes: ny, nz >= 5, max_snap >= 1, Lx, nu > 0, grids given");
    for (int j = 1; j < d->ny; ++j)
        if (!(d->y[j] > d->y[j - 1])) return fail1(nullptr, GKE_ERR_ARG, "y must be strictly increasing");
    for (int j = 1; j < d->nz; ++j)
        if (!(d->z[j] > d->z[j - 1])) return fail1(nullptr, GKE_ERR_ARG, "z must be strictly increasing");
    if (!fft_size_ok(d->nx)) return fail1(nullptr, GKE_ERR_UNSUPPORTED, "nx must be 2^a or 3 * 2^a in [8, 512]");
    if ((long long)d->ny * d->nz > 46340) return fail1(nullptr, GKE_ERR_UNSUPPORTED, "ny nz too large");
    if (d->precision != GKE_PREC_F64 && d->precision != GKE_PREC_F32)
        return fail1(nullptr, d->precision == GKE_PREC_BF16X3 ? GKE_ERR_UNSUPPORTED : GKE_ERR_ARG,
                     "precision must be GKE_PREC_F64 or GKE_PREC_F32");
    gke1h_plan_t p = new gke1h_plan_s;
    p->nx = d->nx; p->ny = d->ny; p->nz = d->nz; p->P = d->ny * d->nz; p->nxh = d->nx / 2 + 1;
    p->max_snap = d->max_snap; p->Lx = d->Lx; p->nu = d->nu; p->st = (cudaStream_t)stream;
    p->f32 = d->precision == GKE_PREC_F32;
    p->npair = (long long)p->P * (p->P + 1) / 2;
    p->nt = (p->P + CT - 1) / CT;
    const size_t cz = p->f32 ? 8 : 16;          // bytes of a complex operand or spectrum value
    const size_t need = cz * p->nxh * ((size_t)8 * p->npair + (size_t)NFLD * p->max_snap * p->P) +
                        (size_t)16 * 4 * p->P * p->nxh * p->max_snap;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    if (need > fr) {
        free_plan(p);
        return fail1(nullptr, GKE_ERR_OOM, "workspaces need " + std::to_string(need >> 20) + " MiB, " +
                                               std::to_string(fr >> 20) + " MiB free");
    }
    // host tables: stencil weights (gke_fd_weights: Fornberg's recursion), twiddles, pair labels
    std::vector<double> wy(5 * p->ny), wz(5 * p->nz);
    std::vector<int> ly(p->ny), lz(p->nz);
    for (int j = 0; j < p->ny; ++j) ly[j] = gke_fd_weights(d->y, p->ny, j, wy.data() + 5 * j);
    for (int j = 0; j < p->nz; ++j) lz[j] = gke_fd_weights(d->z, p->nz, j, wz.data() + 5 * j);
    std::vector<zd> tw(p->nx);
    std::vector<zf> twf(p->nx);
    for (int i = 0; i < p->nx; ++i) {
        const double a = -2.0 * M_PI * i / p->nx;
        tw[i].x = std::cos(a); tw[i].y = std::sin(a);
        twf[i].x = (float)tw[i].x; twf[i].y = (float)tw[i].y;
    }
    std::vector<int> pq(2 * p->npair);
    {
        long long k = 0;
        for (int a = 0; a < p->P; ++a)
            for (int b = a; b < p->P; ++b) { pq[2 * k] = a; pq[2 * k + 1] = b; ++k; }
    }
    std::vector<Job> js;
    make_jobs(js);
    gke_status s = GKE_OK;
    auto al = [&](void** ptr, size_t bytes) {
        if (s != GKE_OK) return;
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); s = fail1(p, GKE_ERR_OOM, "cudaMalloc failed"); }
    };
    al((void**)&p->wy, sizeof(double) * wy.size());
    al((void**)&p->wz, sizeof(double) * wz.size());
    al((void**)&p->ly, sizeof(int) * ly.size());
    al((void**)&p->lz, sizeof(int) * lz.size());
    al((void**)&p->tw, sizeof(zd) * tw.size());
    al((void**)&p->twf, sizeof(zf) * twf.size());
    al((void**)&p->pq, sizeof(int) * pq.size());
    al((void**)&p->prof, sizeof(double) * NPR * p->P);
    al((void**)&p->m1, sizeof(double) * NM1 * p->P);
    al((void**)&p->op, sizeof(double) * NOP * p->P);
    if (p->f32) al((void**)&p->pf, sizeof(float) * R_EPS * p->P);
    al((void**)&p->bad, sizeof(int));
    al(&p->X, cz * (size_t)NFLD * p->nxh * p->max_snap * p->P);
    al(&p->spec, cz * (size_t)(NACC + 1) * p->nxh * p->npair);
    al((void**)&p->fin, sizeof(zd) * (size_t)4 * p->P * p->nxh * p->max_snap);
    if (s != GKE_OK) { std::string m = p->err; free_plan(p); return fail1(nullptr, s, m); }
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (s != GKE_OK) return;
        if (cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError(); s = GKE_ERR_CUDA;
        }
    };
    up(p->wy, wy.data(), sizeof(double) * wy.size());
    up(p->wz, wz.data(), sizeof(double) * wz.size());
    up(p->ly, ly.data(), sizeof(int) * ly.size());
    up(p->lz, lz.data(), sizeof(int) * lz.size());
    up(p->tw, tw.data(), sizeof(zd) * tw.size());
    up(p->twf, twf.data(), sizeof(zf) * twf.size());
    up(p->pq, pq.data(), sizeof(int) * pq.size());
    if (s == GKE_OK && cudaMemcpyToSymbol(c_job, js.data(), sizeof(Job) * NJ) != cudaSuccess) {
        cudaGetLastError(); s = GKE_ERR_CUDA;
    }
    if (s != GKE_OK) { free_plan(p); return fail1(nullptr, s, "uploading the plan's tables failed"); }
    p->smem_prod = (int)(sizeof(zd) * (14 * p->nx + p->nx));
    p->NB = std::max(1, 2048 / p->nx);
    if ((p->f32 ? set_attrs<float>(p) : set_attrs<double>(p)) != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return fail1(nullptr, GKE_ERR_CUDA, "shared-memory attributes refused");
    }
    *out = p;
    return GKE_OK;
}

struct Scope1 {
    gke1h_plan_t p; int stage; cudaEvent_t a = nullptr;
    Scope1(gke1h_plan_t p_, int s) : p(p_), stage(s) {
        if (p->timing) { cudaEventCreate(&a); cudaEventRecord(a, p->st); }
    }
    ~Scope1() {
        if (p->timing && a) {
            cudaEvent_t b;
            cudaEventCreate(&b);
            cudaEventRecord(b, p->st);
            p->marks.push_back({stage, a, b});
        }
    }
};

// every launch of one evaluation, operands / spectra / terms in TF
template <typename TF>
static void launch_pass(gke1h_plan_t p, const zd* f, int ns, TF* T)
{
    typedef cplx<TF> C;
    const int P = p->P, nx = p->nx, nxh = p->nxh;
    const double kx0 = 2.0 * M_PI / p->Lx;
    C* X = (C*)p->X;
    C* spec = (C*)p->spec;
    const C* tw = (const C*)(sizeof(TF) == 8 ? (const void*)p->tw : (const void*)p->twf);
    const TF* pt = (const TF*)(sizeof(TF) == 8 ? (const void*)p->prof : (const void*)p->pf);
    {
        Scope1 sc(p, GKE_STAGE_MEAN);
        k1_mean<<<(P + 127) / 128, 128, 0, p->st>>>(f, ns, P, nxh, p->prof);
        k1_grad<<<(P + 127) / 128, 128, 0, p->st>>>(p->ny, p->nz, p->wy, p->ly, p->wz, p->lz, p->prof, p->pf);
        p->launches += 2;
    }
    {
        Scope1 sc(p, GKE_STAGE_PRODUCTS);
        k1_products<TF><<<P, 256, p->smem_prod, p->st>>>(f, ns, P, nx, p->tw, p->prof, X, p->m1, p->bad);
        k1_onepoint<TF><<<P, 128, 0, p->st>>>(X, ns, p->ny, p->nz, nx, kx0, p->nu, p->wy, p->ly, p->wz, p->lz,
                                             p->m1, p->prof, p->op);
        p->launches += 2;
        if (sizeof(TF) == 4) {
            k1_kgrad<<<(P + 127) / 128, 128, 0, p->st>>>(p->ny, p->nz, p->wy, p->ly, p->wz, p->lz, p->op);
            p->launches += 1;
        }
    }
    {
        Scope1 sc(p, GKE_STAGE_CORRELATE);
        const int nfull = P / CT, rem = P - nfull * CT;
        const bool strips = nfull > 0 && rem > 0 && rem <= STRIP_MAX;
        const int nt = strips ? nfull : p->nt;
        const long long ntp = (long long)nt * (nt + 1) / 2;
        k1_correlate<TF><<<dim3((unsigned)ntp, nxh), 256, 0, p->st>>>(X, ns, P, nx, nt, kx0, p->nu, pt, p->op,
                                                                      spec, p->npair);
        p->launches += 1;
        if (strips) {
            const int cov = nfull * CT;
            const long long n = ((long long)rem * cov + (long long)rem * (rem + 1) / 2) * nxh;
            k1_correlate_strip<TF><<<(unsigned)((n + 127) / 128), 128, 0, p->st>>>(X, ns, P, nx, cov, kx0, p->nu,
                                                                                  pt, p->op, spec, p->npair);
            p->launches += 1;
        }
    }
    {
        Scope1 sc(p, GKE_STAGE_TERMS);
        if (p->reg_tr) {
            const int n2 = nx == 128 ? 8 : 16;
            const long long per = 2LL * (256 / n2);     // pairs per CTA
            const dim3 g((unsigned)((p->npair + per - 1) / per), GKE1H_NTERM);
            if (nx == 128) k1_transform_r<TF, 16, 8><<<g, 256, p->smem_tr, p->st>>>(spec, p->npair, tw, T);
            else if (nx == 256) k1_transform_r<TF, 16, 16><<<g, 256, p->smem_tr, p->st>>>(spec, p->npair, tw, T);
            else k1_transform_r<TF, 32, 16><<<g, 256, p->smem_tr, p->st>>>(spec, p->npair, tw, T);
        } else {
            const long long nblk = (p->npair + 2 * p->NB - 1) / (2 * p->NB);
            k1_transform<TF><<<dim3((unsigned)nblk, GKE1H_NTERM), 256, p->smem_tr, p->st>>>(spec, nx, p->npair,
                                                                                         p->NB, tw, T);
        }
        p->launches += 1;
    }
    {
        Scope1 sc(p, GKE_STAGE_STENCIL);
        Sten S{p->wy, p->ly, p->wz, p->lz, p->ny, p->nz};
        const int G = nx >= 64 ? 4 : 256 / nx;
        const unsigned grid = (unsigned)((p->npair + G - 1) / G);
        k1_stencil_a<TF><<<grid, 256, 0, p->st>>>(T, p->pq, S, nx, p->npair, p->nu);
        k1_stencil_res<TF><<<grid, 256, 0, p->st>>>(T, p->pq, S, nx, p->npair);
        p->launches += 2;
        if (sizeof(TF) == 4) {
            const int Go = nx >= 64 ? 12 : 256 / nx;
            k1_offsets<TF><<<(unsigned)((p->npair + Go - 1) / Go), 256, 0, p->st>>>(T, p->pq, S, nx, p->npair,
                                                                                   p->prof, p->op, p->nu);
            p->launches += 1;
        }
    }
}

extern "C" gke_status gke1h_compute(gke1h_plan_t p, const void* fields, int nsnap, void* terms, double* profiles)
{
    if (!p) return fail1(nullptr, GKE_ERR_ARG, "NULL plan");
    if (!fields || !terms) return fail1(p, GKE_ERR_ARG, "NULL fields or terms");
    if (nsnap < 1 || nsnap > p->max_snap) return fail1(p, GKE_ERR_ARG, "nsnap outside [1, max_snap]");
    const int P = p->P, nx = p->nx, nxh = p->nxh, ns = nsnap;
    const size_t fbytes = sizeof(zd) * (size_t)ns * 4 * P * nxh;
    const size_t tbytes = (p->f32 ? 4 : 8) * (size_t)GKE1H_NTERM * p->npair * nx;
    const zd* f = (const zd*)fields;
    if (!on_device(fields)) {
        TRY1(p, cudaMemcpyAsync(p->fin, fields, fbytes, cudaMemcpyHostToDevice, p->st));
        f = p->fin;
    }
    const bool dev_out = on_device(terms);
    void* T = terms;
    if (!dev_out) {
        if (!p->terms) TRY1(p, cudaMalloc(&p->terms, tbytes));
        T = p->terms;
    }
    TRY1(p, cudaMemsetAsync(p->bad, 0, sizeof(int), p->st));
    if (p->f32) launch_pass<float>(p, f, ns, (float*)T);
    else launch_pass<double>(p, f, ns, (double*)T);
    TRY1(p, cudaGetLastError());
    if (!dev_out) TRY1(p, cudaMemcpyAsync(terms, T, tbytes, cudaMemcpyDeviceToHost, p->st));
    if (profiles)
        TRY1(p, cudaMemcpyAsync(profiles, p->prof, sizeof(double) * GKE1H_NPROF * P,
                                on_device(profiles) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->st));
    int bad = 0;
    TRY1(p, cudaMemcpyAsync(&bad, p->bad, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    TRY1(p, cudaStreamSynchronize(p->st));
    if (bad) return fail1(p, GKE_ERR_NONFINITE, "the input holds a NaN or Inf");
    return GKE_OK;
}

extern "C" long long gke1h_npair(gke1h_plan_t p) { return p ? p->npair : -1; }

extern "C" long long gke1h_pair_labels(int ny, int nz, const double* y, const double* z, int* p1, int* p2,
                                       double* Y1, double* Z1, double* Y2, double* Z2)
{
    if (!y || !z || ny < 1 || nz < 1) return -1;
    const long long P = (long long)ny * nz;
    long long k = 0;
    for (long long a = 0; a < P; ++a)
        for (long long b = a; b < P; ++b, ++k) {
            if (p1) p1[k] = (int)a;
            if (p2) p2[k] = (int)b;
            if (Y1) Y1[k] = y[a / nz];
            if (Z1) Z1[k] = z[a % nz];
            if (Y2) Y2[k] = y[b / nz];
            if (Z2) Z2[k] = z[b % nz];
        }
    return k;
}

extern "C" gke_status gke1h_set_timing(gke1h_plan_t p, int on)
{
    if (!p) return GKE_ERR_ARG;
    p->timing = on != 0;
    return GKE_OK;
}

extern "C" gke_status gke1h_stage_times(gke1h_plan_t p, double* ms)
{
    if (!p || !ms) return p ? fail1(p, GKE_ERR_ARG, "ms is NULL") : GKE_ERR_ARG;
    TRY1(p, cudaStreamSynchronize(p->st));
    for (int i = 0; i < GKE_NSTAGE; ++i) ms[i] = 0.0;
    for (auto& m : p->marks) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) ms[m.stage] += t;
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    p->marks.clear();
    return GKE_OK;
}

extern "C" long long gke1h_launch_count(gke1h_plan_t p) { return p ? p->launches : -1; }

extern "C" const char* gke1h_last_error(gke1h_plan_t p) { return p ? p->err.c_str() : g1_err.c_str(); }

extern "C" void gke1h_destroy(gke1h_plan_t p) { free_plan(p); }
