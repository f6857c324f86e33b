// gke1h.cu -- the GKE for a flow with one homogeneous direction (x): plan,
// kernels and the C ABI of include/gke1h.h.
//
// The paper's method (Sec. 3) with Parseval in x only and the second
// inhomogeneous direction z handled like the wall-normal one (Sec. 5): every
// pair of cross-section points (p1, p2) plays the part of a (Y1, Y2) pair.
// Stages of one evaluation, all FP64:
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
using gke::mk;

namespace gke1h {

// operand fields: the fluctuations and the in-plane products
enum Fld { G_U = 0, G_V, G_W, G_P, G_Q, G_UU, G_UV, G_UW, G_VV, G_VW, G_WW, NFLD };
// per-pair term accumulators (the residual is formed at the end)
enum Acc { A_A = 0, A_PHIX, A_PHIY, A_PHIZ, A_PSIY, A_PSIZ, A_XI, NACC };
// one-point sums per point: <u_i u_j> (uu vv ww uv uw vw), <q u_k>, <p v>, <p w>
enum M1 { M_UU = 0, M_VV, M_WW, M_UV, M_UW, M_VW, M_QU, M_QV, M_QW, M_PV, M_PW, NM1 };
// one-point parts of the terms per point: K = <u_i u_i>, <q u_k>, <p u_k>, 2 (Pi - eps)
enum OP { O_K = 0, O_SX, O_SY, O_SZ, O_PY, O_PZ, O_E0, NOP };
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
__global__ void k1_grad(int ny, int nz, const double* __restrict__ wy, const int* __restrict__ ly,
                        const double* __restrict__ wz, const int* __restrict__ lz, double* __restrict__ prof)
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
}

// --------------------------------------------------------------- products
// One CTA per point p.  Shared memory: two buffers of NFLD - 4 = 7
// sequences of nx complex values and the nx twiddles.  Thread t owns the
// physical points x = t, t + blockDim, ... (at most two: nx <= 512).
__global__ void __launch_bounds__(256)
k1_products(const zd* __restrict__ f, int ns, int P, int nx, const zd* __restrict__ tw,
            const double* __restrict__ prof, zd* __restrict__ X, double* __restrict__ m1, int* __restrict__ bad)
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
            X[(((long long)c * nxh + m) * ns + s) * P + p] = v;
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
            X[(((long long)(G_Q + j) * nxh + m) * ns + s) * P + p] = mk(v.x * inv_nx, v.y * inv_nx);
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
__global__ void __launch_bounds__(128)
k1_onepoint(const zd* __restrict__ X, int ns, int ny, int nz, int nx, double kx0, double nu,
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
        const zd* row = X + (((long long)i * nxh + m) * ns + s) * P;
        const zd a = row[p];
        zd dy = mk(0.0, 0.0), dz = mk(0.0, 0.0);
        for (int l = 0; l < 5; ++l) {
            const zd t1 = row[(ly[iy] + l) * nz + iz], t2 = row[iy * nz + lz[iz] + l];
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

// -------------------------------------------------------------- correlate
#define CT 32        // tile edge (points)
#define SCH 8        // snapshots per shared-memory chunk
#define STRIP_MAX 8  // widest remainder past the last full tile done as strips

__device__ __forceinline__ void cmac(zd& acc, const zd a, const zd b)     // acc += conj(a) b
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

// add contraction jb's value at (q1, q2) into the accumulators of that pair
__device__ __forceinline__ void add_job(zd* T, const Job& jb, const zd acc, int q1, int q2, int P,
                                        const double* __restrict__ prof)
{
    #pragma unroll
    for (int t = 0; t < 6; ++t) {
        const double c = jb.c[t];
        if (c == 0.0) continue;
        T[t].x = fma(c, acc.x, T[t].x);
        T[t].y = fma(c, acc.y, T[t].y);
    }
    if (jb.ra >= 0) {
        // xi: <u_a(p1) u_b(p2)'> enters -2 <du_i du_k> (d_k U_i)* - 2 <du_i u_k*> d(d_k U_i)
        // with weight 2 d_b U_a(p2) (b = y, z) + 2 d_a U_b(p1) (a = y, z)
        const int ra = jb.ra, rb = jb.rb;
        double c = 0.0;
        if (rb >= 1 && q2 < P) c += 2.0 * prof[(long long)(R_G + 2 * ra + rb - 1) * P + q2];
        if (ra >= 1 && q1 < P) c += 2.0 * prof[(long long)(R_G + 2 * rb + ra - 1) * P + q1];
        T[A_XI].x = fma(c, acc.x, T[A_XI].x);
        T[A_XI].y = fma(c, acc.y, T[A_XI].y);
    }
}

// snapshot average, one-point parts (m = 0), mean-flow couplings and the
// residual's spectral part; writes the eight spectra of pair (q1 <= q2)
__device__ __forceinline__ void finish_pair(const zd* T, int q1, int q2, int m, int nx, double kx0, double nu,
                                            int ns, int P, const double* __restrict__ prof,
                                            const double* __restrict__ op, zd* __restrict__ spec, long long npair)
{
    const int nxh = nx / 2 + 1;
    const double inv = 1.0 / ns;
    const double k = (2 * m == nx) ? 0.0 : kx0 * m;
    zd v[NACC];
    #pragma unroll
    for (int t = 0; t < NACC; ++t) v[t] = mk(T[t].x * inv, T[t].y * inv);
    auto O = [&](int r, int q) { return op[(long long)r * P + q]; };
    auto U = [&](int r, int q) { return prof[(long long)r * P + q]; };
    if (m == 0) {
        v[A_A].x += O(O_K, q1) + O(O_K, q2);
        v[A_PHIX].x += O(O_SX, q2) - O(O_SX, q1);
        v[A_PHIY].x += O(O_SY, q2) - O(O_SY, q1);
        v[A_PHIZ].x += O(O_SZ, q2) - O(O_SZ, q1);
        v[A_PSIY].x += 0.5 * (O(O_SY, q1) + O(O_SY, q2)) + 2.0 * (O(O_PY, q1) + O(O_PY, q2));
        v[A_PSIZ].x += 0.5 * (O(O_SZ, q1) + O(O_SZ, q2)) + 2.0 * (O(O_PZ, q1) + O(O_PZ, q2));
        v[A_XI].x += O(O_E0, q1) + O(O_E0, q2);
    }
    const zd A = v[A_A];
    const double dU = U(R_U, q2) - U(R_U, q1), dV = U(R_V, q2) - U(R_V, q1), dW = U(R_W, q2) - U(R_W, q1);
    const double Vs = 0.5 * (U(R_V, q1) + U(R_V, q2)), Ws = 0.5 * (U(R_W, q1) + U(R_W, q2));
    // Phi_x += dU A - 2 nu (i k) A
    v[A_PHIX].x += dU * A.x + 2.0 * nu * k * A.y;
    v[A_PHIX].y += dU * A.y - 2.0 * nu * k * A.x;
    v[A_PHIY].x += dV * A.x; v[A_PHIY].y += dV * A.y;
    v[A_PHIZ].x += dW * A.x; v[A_PHIZ].y += dW * A.y;
    v[A_PSIY].x += Vs * A.x; v[A_PSIY].y += Vs * A.y;
    v[A_PSIZ].x += Ws * A.x; v[A_PSIZ].y += Ws * A.y;
    // residual spectrum: i k Phi_x - xi (the stencil parts come later)
    const zd res = mk(-k * v[A_PHIX].y - v[A_XI].x, k * v[A_PHIX].x - v[A_XI].y);
    const long long pr = tri(q1, q2, P);
    #pragma unroll
    for (int t = 0; t < NACC; ++t) spec[((long long)t * nxh + m) * npair + pr] = v[t];
    spec[((long long)NACC * nxh + m) * npair + pr] = res;
}

// CTA = (tile pair T1 <= T2 of the nt full tiles, wavenumber m); 16 x 16
// threads, each an RB x RB block of pairs (p1 = T1 CT + ty + 16 a,
// p2 = T2 CT + tx + 16 b).  With strips, the points past the last full tile
// are left to k1_correlate_strip; otherwise the last tile is padded.
__global__ void __launch_bounds__(256, 1)
k1_correlate(const zd* __restrict__ X, int ns, int P, int nx, int nt, double kx0, double nu,
             const double* __restrict__ prof, const double* __restrict__ op, zd* __restrict__ spec, long long npair)
{
    constexpr int RB = 2;
    __shared__ zd As[SCH][CT];
    __shared__ zd Bs[SCH][CT];
    const int nxh = nx / 2 + 1;
    const int m = blockIdx.y;
    int T1 = 0, rem = blockIdx.x;
    while (rem >= nt - T1) { rem -= nt - T1; ++T1; }
    const int T2 = T1 + rem;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int p1[RB], p2[RB];
    for (int a = 0; a < RB; ++a) { p1[a] = T1 * CT + ty + 16 * a; p2[a] = T2 * CT + tx + 16 * a; }
    zd T[NACC][RB][RB];
    #pragma unroll
    for (int t = 0; t < NACC; ++t)
        #pragma unroll
        for (int a = 0; a < RB; ++a)
            #pragma unroll
            for (int b = 0; b < RB; ++b) T[t][a][b] = mk(0.0, 0.0);
    for (int j = 0; j < NJ; ++j) {
        const Job& jb = c_job[j];
        zd acc[RB][RB];
        #pragma unroll
        for (int a = 0; a < RB; ++a)
            #pragma unroll
            for (int b = 0; b < RB; ++b) acc[a][b] = mk(0.0, 0.0);
        for (int t = 0; t < jb.nt; ++t) {
            const double wt = jb.w[t];
            const zd* A = X + ((long long)jb.fa[t] * nxh + m) * ns * P;
            const zd* B = X + ((long long)jb.fb[t] * nxh + m) * ns * P;
            zd part[RB][RB];
            #pragma unroll
            for (int a = 0; a < RB; ++a)
                #pragma unroll
                for (int b = 0; b < RB; ++b) part[a][b] = mk(0.0, 0.0);
            for (int s0 = 0; s0 < ns; s0 += SCH) {
                __syncthreads();
                for (int e = threadIdx.x; e < SCH * CT; e += blockDim.x) {
                    const int ss = e / CT, yy = e - ss * CT, s = s0 + ss;
                    zd va = mk(0.0, 0.0), vb = mk(0.0, 0.0);
                    if (s < ns && T1 * CT + yy < P) va = A[(long long)s * P + T1 * CT + yy];
                    if (s < ns && T2 * CT + yy < P) vb = B[(long long)s * P + T2 * CT + yy];
                    As[ss][yy] = va;
                    Bs[ss][yy] = vb;
                }
                __syncthreads();
                #pragma unroll
                for (int ss = 0; ss < SCH; ++ss) {
                    zd av[RB], bv[RB];
                    #pragma unroll
                    for (int i = 0; i < RB; ++i) { av[i] = As[ss][ty + 16 * i]; bv[i] = Bs[ss][tx + 16 * i]; }
                    #pragma unroll
                    for (int a = 0; a < RB; ++a)
                        #pragma unroll
                        for (int b = 0; b < RB; ++b) cmac(part[a][b], av[a], bv[b]);
                }
            }
            #pragma unroll
            for (int a = 0; a < RB; ++a)
                #pragma unroll
                for (int b = 0; b < RB; ++b) {
                    acc[a][b].x = fma(wt, part[a][b].x, acc[a][b].x);
                    acc[a][b].y = fma(wt, part[a][b].y, acc[a][b].y);
                }
        }
        // the contraction into the term spectra (as add_job, one coefficient test per job)
        #pragma unroll
        for (int t = 0; t < 6; ++t) {
            const double c = jb.c[t];
            if (c == 0.0) continue;
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
                    double c = 0.0;
                    if (rb >= 1 && p2[b] < P) c += 2.0 * prof[(long long)(R_G + 2 * ra + rb - 1) * P + p2[b]];
                    if (ra >= 1 && p1[a] < P) c += 2.0 * prof[(long long)(R_G + 2 * rb + ra - 1) * P + p1[a]];
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
            zd v[NACC];
            #pragma unroll
            for (int t = 0; t < NACC; ++t) v[t] = T[t][a][b];
            finish_pair(v, p1[a], p2[b], m, nx, kx0, nu, ns, P, prof, op, spec, npair);
        }
}

// The pairs (p1 <= p2) with p2 >= cov (the points past the last full tile):
// one thread per (pair, wavenumber), the same contractions one pair at a time;
// consecutive threads take consecutive p1 (coalesced operand loads).
__global__ void __launch_bounds__(128)
k1_correlate_strip(const zd* __restrict__ X, int ns, int P, int nx, int cov, double kx0, double nu,
                   const double* __restrict__ prof, const double* __restrict__ op, zd* __restrict__ spec,
                   long long npair)
{
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
    zd T[NACC];
    #pragma unroll
    for (int t = 0; t < NACC; ++t) T[t] = mk(0.0, 0.0);
    for (int j = 0; j < NJ; ++j) {
        const Job& jb = c_job[j];
        zd acc = mk(0.0, 0.0);
        for (int t = 0; t < jb.nt; ++t) {
            const zd* A = X + ((long long)jb.fa[t] * nxh + m) * ns * P;
            const zd* B = X + ((long long)jb.fb[t] * nxh + m) * ns * P;
            zd part = mk(0.0, 0.0);
            for (int s = 0; s < ns; ++s) cmac(part, A[(long long)s * P + q1], B[(long long)s * P + q2]);
            acc.x = fma(jb.w[t], part.x, acc.x);
            acc.y = fma(jb.w[t], part.y, acc.y);
        }
        add_job(T, jb, acc, q1, q2, P, prof);
    }
    finish_pair(T, q1, q2, m, nx, kx0, nu, ns, P, prof, op, spec, npair);
}

// ------------------------------------------------------------- transforms
// CTA = 2 NB consecutive pairs of one term.  The spectra (nx/2 + 1
// wavenumbers each, imaginary parts dropped at m = 0 and m = nx/2) are
// staged in shared memory; pairs 2b and 2b + 1 share one complex sequence,
// H_2b + i H_2b+1 with H the Hermitian extension, whose inverse transform
// has the two real correlations as its real and imaginary parts.
__global__ void __launch_bounds__(256)
k1_transform(const zd* __restrict__ spec, int nx, long long npair, int NB, const zd* __restrict__ tw,
             double* __restrict__ terms)
{
    extern __shared__ zd sm[];
    const int nxh = nx / 2 + 1;
    zd* b0 = sm;
    zd* b1 = sm + (size_t)NB * nx;
    zd* stw = sm + (size_t)2 * NB * nx;
    zd* stg = stw + nx;                               // [2 NB][nxh]
    gke::load_twiddles(stw, tw, nx);
    const int t = blockIdx.y;
    const long long pr0 = (long long)blockIdx.x * 2 * NB;
    const int np = (int)std::min<long long>(2 * NB, npair - pr0);
    for (int e = threadIdx.x; e < nxh * 2 * NB; e += blockDim.x) {
        const int m = e / (2 * NB), c = e - m * 2 * NB;
        zd v = mk(0.0, 0.0);
        if (c < np) v = spec[((long long)t * nxh + m) * npair + pr0 + c];
        if (m == 0 || 2 * m == nx) v.y = 0.0;
        stg[c * nxh + m] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NB * nx; e += blockDim.x) {
        const int b = e / nx, k = e - b * nx;
        const bool lo = 2 * k <= nx;
        const zd a = stg[(2 * b) * nxh + (lo ? k : nx - k)];
        const zd c = stg[(2 * b + 1) * nxh + (lo ? k : nx - k)];
        const double ay = lo ? a.y : -a.y, cy = lo ? c.y : -c.y;
        b0[b * nx + k] = mk(a.x - cy, ay + c.x);
    }
    zd* r = gke::fft_block<double, true>(b0, b1, nx, NB, nx, stw);
    for (int e = threadIdx.x; e < np * nx; e += blockDim.x) {
        const int c = e / nx, x = e - c * nx;
        const zd z = r[(c >> 1) * nx + x];
        terms[((long long)t * npair + pr0 + c) * nx + x] = (c & 1) ? z.y : z.x;
    }
}

// Register-FFT variant for nx = N1 N2 (gke::fft2l, twiddles resolved at
// compile time): CTA = RZ sequences x N2 lanes, each sequence two pairs
// packed as above; lane l holds the wavenumbers l + N2 j of its sequence.
template <int N1, int N2>
__global__ void __launch_bounds__(256)
k1_transform_r(const zd* __restrict__ spec, long long npair, const zd* __restrict__ tw, double* __restrict__ terms)
{
    constexpr int N = N1 * N2, nxh = N / 2 + 1, RZ = 256 / N2;
    extern __shared__ zd sm[];
    zd* stw = sm;
    zd* xs = sm + N;
    const int lane = threadIdx.x % N2, r = threadIdx.x / N2;
    const int t = blockIdx.y;
    const long long pa = ((long long)blockIdx.x * RZ + r) * 2, pb = pa + 1;
    const bool la = pa < npair, lb = pb < npair;
    gke::load_twiddles(stw, tw, N);
    // spectra [t][m][pair]: the two pairs of a sequence share 32-byte sectors
    const zd* sa = spec + (long long)t * nxh * npair + (la ? pa : 0);
    const zd* sb = spec + (long long)t * nxh * npair + (lb ? pb : 0);
    zd v[N1];
    #pragma unroll
    for (int j = 0; j < N1; ++j) {
        const int k = lane + N2 * j;
        const bool lo = 2 * k <= N;
        zd a = mk(0.0, 0.0), b = a;
        if (la) { a = sa[(long long)(lo ? k : N - k) * npair]; if (!lo) a.y = -a.y; }
        if (lb) { b = sb[(long long)(lo ? k : N - k) * npair]; if (!lo) b.y = -b.y; }
        if (k == 0 || 2 * k == N) { a.y = 0.0; b.y = 0.0; }
        v[j] = mk(a.x - b.y, a.y + b.x);
    }
    __syncthreads();                                  // twiddles staged
    gke::fft2l<double, N1, N2, true>(v, lane, xs + r * N1 * (N2 + 1), N2 + 1, 1, stw);
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

__device__ __forceinline__ void neighbours(const Sten& S, const int* __restrict__ pq, long long pr0, int G,
                                           int nx, long long npair, long long (*off)[20], signed char (*flip)[20],
                                           double (*w)[20])
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
        w[g][j] = wt;
    }
    __syncthreads();
}

// d_Y1, d_Y2, d_Z1, d_Z2 of one plane at separation m of CTA pair g
__device__ __forceinline__ void derivs4(const double* __restrict__ plane, const long long* off,
                                        const signed char* flip, const double* w, int m, int nx, double sg,
                                        double d[4])
{
    const int mm = m == 0 ? 0 : nx - m;
    #pragma unroll
    for (int dir = 0; dir < 4; ++dir) {
        double acc = 0.0;
        #pragma unroll
        for (int l = 0; l < 5; ++l) {
            const int j = 5 * dir + l;
            const double v = flip[j] ? sg * plane[off[j] + mm] : plane[off[j] + m];
            acc = fma(w[j], v, acc);
        }
        d[dir] = acc;
    }
}

__global__ void __launch_bounds__(256)
k1_stencil_a(double* __restrict__ terms, const int* __restrict__ pq, Sten S, int nx, long long npair, double nu)
{
    __shared__ long long off[SG][20];
    __shared__ signed char flip[SG][20];
    __shared__ double w[SG][20];
    const int G = nx >= 64 ? 4 : 256 / nx;
    const long long pr0 = (long long)blockIdx.x * G;
    neighbours(S, pq, pr0, G, nx, npair, off, flip, w);
    const double* Ap = terms + (long long)GKE1H_TERM_A * npair * nx;
    for (int e = threadIdx.x; e < G * nx; e += blockDim.x) {
        const int g = e / nx, m = e - g * nx;
        const long long pr = pr0 + g;
        if (pr >= npair) continue;
        double d[4];
        derivs4(Ap, off[g], flip[g], w[g], m, nx, 1.0, d);
        terms[((long long)GKE1H_TERM_PHI_Y * npair + pr) * nx + m] -= nu * (d[1] - d[0]);
        terms[((long long)GKE1H_TERM_PHI_Z * npair + pr) * nx + m] -= nu * (d[3] - d[2]);
        terms[((long long)GKE1H_TERM_PSI_Y * npair + pr) * nx + m] -= 0.5 * nu * (d[0] + d[1]);
        terms[((long long)GKE1H_TERM_PSI_Z * npair + pr) * nx + m] -= 0.5 * nu * (d[2] + d[3]);
    }
}

__global__ void __launch_bounds__(256)
k1_stencil_res(double* __restrict__ terms, const int* __restrict__ pq, Sten S, int nx, long long npair)
{
    __shared__ long long off[SG][20];
    __shared__ signed char flip[SG][20];
    __shared__ double w[SG][20];
    const int G = nx >= 64 ? 4 : 256 / nx;
    const long long pr0 = (long long)blockIdx.x * G;
    neighbours(S, pq, pr0, G, nx, npair, off, flip, w);
    auto plane = [&](int t) { return terms + (long long)t * npair * nx; };
    for (int e = threadIdx.x; e < G * nx; e += blockDim.x) {
        const int g = e / nx, m = e - g * nx;
        const long long pr = pr0 + g;
        if (pr >= npair) continue;
        double fy[4], fz[4], sy[4], sz[4];
        derivs4(plane(GKE1H_TERM_PHI_Y), off[g], flip[g], w[g], m, nx, -1.0, fy);
        derivs4(plane(GKE1H_TERM_PHI_Z), off[g], flip[g], w[g], m, nx, -1.0, fz);
        derivs4(plane(GKE1H_TERM_PSI_Y), off[g], flip[g], w[g], m, nx, 1.0, sy);
        derivs4(plane(GKE1H_TERM_PSI_Z), off[g], flip[g], w[g], m, nx, 1.0, sz);
        terms[((long long)GKE1H_TERM_RESIDUAL * npair + pr) * nx + m] +=
            0.5 * (fy[1] - fy[0]) + 0.5 * (fz[3] - fz[2]) + (sy[0] + sy[1]) + (sz[2] + sz[3]);
    }
}

}  // namespace gke1h

// =================================================================== plan
using namespace gke1h;

struct gke1h_plan_s {
    int nx = 0, ny = 0, nz = 0, P = 0, nxh = 0, max_snap = 0, nt = 0;
    long long npair = 0;
    double Lx = 0, nu = 0;
    cudaStream_t st = nullptr;
    double *wy = nullptr, *wz = nullptr, *prof = nullptr, *m1 = nullptr, *op = nullptr, *terms = nullptr;
    int *ly = nullptr, *lz = nullptr, *pq = nullptr, *bad = nullptr;
    zd *tw = nullptr, *X = nullptr, *spec = nullptr, *fin = nullptr;
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
                    p->tw, p->X, p->spec, p->fin};
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
    gke1h_plan_t p = new gke1h_plan_s;
    p->nx = d->nx; p->ny = d->ny; p->nz = d->nz; p->P = d->ny * d->nz; p->nxh = d->nx / 2 + 1;
    p->max_snap = d->max_snap; p->Lx = d->Lx; p->nu = d->nu; p->st = (cudaStream_t)stream;
    p->npair = (long long)p->P * (p->P + 1) / 2;
    p->nt = (p->P + CT - 1) / CT;
    const size_t need = (size_t)16 * p->nxh * ((size_t)8 * p->npair + (size_t)NFLD * p->max_snap * p->P) +
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
    for (int i = 0; i < p->nx; ++i) {
        const double a = -2.0 * M_PI * i / p->nx;
        tw[i].x = std::cos(a); tw[i].y = std::sin(a);
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
    al((void**)&p->pq, sizeof(int) * pq.size());
    al((void**)&p->prof, sizeof(double) * NPR * p->P);
    al((void**)&p->m1, sizeof(double) * NM1 * p->P);
    al((void**)&p->op, sizeof(double) * NOP * p->P);
    al((void**)&p->bad, sizeof(int));
    al((void**)&p->X, sizeof(zd) * (size_t)NFLD * p->nxh * p->max_snap * p->P);
    al((void**)&p->spec, sizeof(zd) * (size_t)(NACC + 1) * p->nxh * p->npair);
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
    up(p->pq, pq.data(), sizeof(int) * pq.size());
    if (s == GKE_OK && cudaMemcpyToSymbol(c_job, js.data(), sizeof(Job) * NJ) != cudaSuccess) {
        cudaGetLastError(); s = GKE_ERR_CUDA;
    }
    if (s != GKE_OK) { free_plan(p); return fail1(nullptr, s, "uploading the plan's tables failed"); }
    p->smem_prod = (int)(sizeof(zd) * (14 * p->nx + p->nx));
    p->NB = std::max(1, 2048 / p->nx);
    p->smem_tr = (int)(sizeof(zd) * (3 * p->NB * p->nx + 2 * p->NB + p->nx));
    cudaError_t ea = cudaSuccess;
    if (p->nx == 128 || p->nx == 256 || p->nx == 512) {
        const void* fn = p->nx == 128 ? (const void*)k1_transform_r<16, 8>
                       : p->nx == 256 ? (const void*)k1_transform_r<16, 16> : (const void*)k1_transform_r<32, 16>;
        const int n2 = p->nx == 128 ? 8 : 16, n1 = p->nx / n2;
        p->smem_tr = (int)(sizeof(zd) * (p->nx + (256 / n2) * n1 * (n2 + 1)));
        ea = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->smem_tr);
        p->reg_tr = true;
    } else {
        ea = cudaFuncSetAttribute(k1_transform, cudaFuncAttributeMaxDynamicSharedMemorySize, p->smem_tr);
    }
    if (cudaFuncSetAttribute(k1_products, cudaFuncAttributeMaxDynamicSharedMemorySize, p->smem_prod) != cudaSuccess ||
        ea != cudaSuccess) {
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

extern "C" gke_status gke1h_compute(gke1h_plan_t p, const void* fields, int nsnap, double* terms, double* profiles)
{
    if (!p) return fail1(nullptr, GKE_ERR_ARG, "NULL plan");
    if (!fields || !terms) return fail1(p, GKE_ERR_ARG, "NULL fields or terms");
    if (nsnap < 1 || nsnap > p->max_snap) return fail1(p, GKE_ERR_ARG, "nsnap outside [1, max_snap]");
    const int P = p->P, nx = p->nx, nxh = p->nxh, ns = nsnap;
    const size_t fbytes = sizeof(zd) * (size_t)ns * 4 * P * nxh;
    const zd* f = (const zd*)fields;
    if (!on_device(fields)) {
        TRY1(p, cudaMemcpyAsync(p->fin, fields, fbytes, cudaMemcpyHostToDevice, p->st));
        f = p->fin;
    }
    const bool dev_out = on_device(terms);
    double* T = terms;
    if (!dev_out) {
        if (!p->terms) TRY1(p, cudaMalloc(&p->terms, sizeof(double) * (size_t)GKE1H_NTERM * p->npair * nx));
        T = p->terms;
    }
    const double kx0 = 2.0 * M_PI / p->Lx;
    TRY1(p, cudaMemsetAsync(p->bad, 0, sizeof(int), p->st));
    {
        Scope1 sc(p, GKE_STAGE_MEAN);
        k1_mean<<<(P + 127) / 128, 128, 0, p->st>>>(f, ns, P, nxh, p->prof);
        k1_grad<<<(P + 127) / 128, 128, 0, p->st>>>(p->ny, p->nz, p->wy, p->ly, p->wz, p->lz, p->prof);
        p->launches += 2;
    }
    {
        Scope1 sc(p, GKE_STAGE_PRODUCTS);
        k1_products<<<P, 256, p->smem_prod, p->st>>>(f, ns, P, nx, p->tw, p->prof, p->X, p->m1, p->bad);
        k1_onepoint<<<P, 128, 0, p->st>>>(p->X, ns, p->ny, p->nz, nx, kx0, p->nu, p->wy, p->ly,
                                                        p->wz, p->lz, p->m1, p->prof, p->op);
        p->launches += 2;
    }
    {
        Scope1 sc(p, GKE_STAGE_CORRELATE);
        const int nfull = P / CT, rem = P - nfull * CT;
        const bool strips = nfull > 0 && rem > 0 && rem <= STRIP_MAX;
        const int nt = strips ? nfull : p->nt;
        const long long ntp = (long long)nt * (nt + 1) / 2;
        k1_correlate<<<dim3((unsigned)ntp, nxh), 256, 0, p->st>>>(p->X, ns, P, nx, nt, kx0, p->nu, p->prof,
                                                                  p->op, p->spec, p->npair);
        p->launches += 1;
        if (strips) {
            const int cov = nfull * CT;
            const long long n = ((long long)rem * cov + (long long)rem * (rem + 1) / 2) * nxh;
            k1_correlate_strip<<<(unsigned)((n + 127) / 128), 128, 0, p->st>>>(p->X, ns, P, nx, cov, kx0, p->nu,
                                                                              p->prof, p->op, p->spec, p->npair);
            p->launches += 1;
        }
    }
    {
        Scope1 sc(p, GKE_STAGE_TERMS);
        if (p->reg_tr) {
            const int n2 = nx == 128 ? 8 : 16;
            const long long per = 2LL * (256 / n2);     // pairs per CTA
            const dim3 g((unsigned)((p->npair + per - 1) / per), GKE1H_NTERM);
            if (nx == 128) k1_transform_r<16, 8><<<g, 256, p->smem_tr, p->st>>>(p->spec, p->npair, p->tw, T);
            else if (nx == 256) k1_transform_r<16, 16><<<g, 256, p->smem_tr, p->st>>>(p->spec, p->npair, p->tw, T);
            else k1_transform_r<32, 16><<<g, 256, p->smem_tr, p->st>>>(p->spec, p->npair, p->tw, T);
        } else {
            const long long nblk = (p->npair + 2 * p->NB - 1) / (2 * p->NB);
            k1_transform<<<dim3((unsigned)nblk, GKE1H_NTERM), 256, p->smem_tr, p->st>>>(p->spec, nx, p->npair,
                                                                                     p->NB, p->tw, T);
        }
        p->launches += 1;
    }
    {
        Scope1 sc(p, GKE_STAGE_STENCIL);
        Sten S{p->wy, p->ly, p->wz, p->lz, p->ny, p->nz};
        const int G = nx >= 64 ? 4 : 256 / nx;
        const unsigned grid = (unsigned)((p->npair + G - 1) / G);
        k1_stencil_a<<<grid, 256, 0, p->st>>>(T, p->pq, S, nx, p->npair, p->nu);
        k1_stencil_res<<<grid, 256, 0, p->st>>>(T, p->pq, S, nx, p->npair);
        p->launches += 2;
    }
    TRY1(p, cudaGetLastError());
    if (!dev_out)
        TRY1(p, cudaMemcpyAsync(terms, T, sizeof(double) * (size_t)GKE1H_NTERM * p->npair * nx,
                                cudaMemcpyDeviceToHost, p->st));
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
