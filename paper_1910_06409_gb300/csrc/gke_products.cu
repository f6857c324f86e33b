// gke_products.cu -- Step 1 (ensemble mean) and the per-snapshot part of
// Step 2 that precedes the correlations: fluctuations, the in-plane products
// formed in physical space (Sec. 3.1: widehat{uu} = F(u u)), their forward
// transforms, and the one-point statistics the assembly needs.
//
// Transforms along z act on tiles of adjacent kx columns; transforms along x
// on two real rows at a time (packed as real and imaginary part of one
// complex sequence).  The transform arithmetic runs in TF = double (plain
// path) or float (split path); one-point sums are always FP64.
#include <algorithm>

#include "gke_common.cuh"
#include "gke_kernels.h"

namespace gke {

// ---------------------------------------------------------------- Step 1
// mean_sum[f][y] += sum_s Re f_hat_s(y, k = 0): the (0,0) coefficient is the
// plane mean, so this accumulates the ensemble mean of u, v, w, p (Step 1).
__global__ void k_mean_accum(const zd* __restrict__ fields, int ns, int ny, long long plane,
                             double* __restrict__ mean_sum)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * ny) return;
    int f = idx / ny, y = idx - f * ny;
    double acc = 0.0;
    for (int s = 0; s < ns; ++s) acc += fields[(((long long)s * 4 + f) * ny + y) * plane].x;
    mean_sum[idx] += acc;
}

template <typename TF> __device__ __forceinline__ cplx<TF> cvt(zd v) { return mk((TF)v.x, (TF)v.y); }

// ---------------------------------------------- linear fields -> operands
// Xop[f][k][s][y] = fields[s][f][y][k] - mean_f(y) [k == 0], f = u, v, w, p.
// Tile of 32 wavenumbers x one y chunk (the ny rows split into equal chunks
// of at most ll_rows: 34 KB of shared memory) transposed through shared
// memory in TF; flags non-finite input.
template <typename TF> __host__ __device__ constexpr int ll_rows() { return sizeof(TF) == 4 ? 128 : 64; }
template <typename TF>
__global__ void __launch_bounds__(256)
k_load_linear(const zd* __restrict__ fields, int ns, int ny, int Nk, int rows, int s0,
              const double* __restrict__ mean, cplx<TF>* __restrict__ Xop, int* __restrict__ nonfinite)
{
    __shared__ cplx<TF> tile[ll_rows<TF>()][33];
    const int k0 = blockIdx.x * 32, y0 = blockIdx.y * rows;
    const int s = s0 + blockIdx.z / 4, f = blockIdx.z % 4;
    const int nr = min(rows, ny - y0);
    int bad = 0;
    for (int r = threadIdx.y; r < nr; r += blockDim.y) {
        const int y = y0 + r, k = k0 + threadIdx.x;
        if (k < Nk) {
            zd v = fields[(((long long)s * 4 + f) * ny + y) * Nk + k];
            if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
            if (k == 0) v.x -= mean[f * ny + y];
            tile[r][threadIdx.x] = cvt<TF>(v);
        }
    }
    if (bad) atomicOr(nonfinite, 1);
    __syncthreads();
    for (int kk = threadIdx.y; kk < 32; kk += blockDim.y) {
        const int k = k0 + kk;
        if (k >= Nk) break;
        cplx<TF>* dst = Xop + (((long long)f * Nk + k) * ns + s) * ny + y0;
        for (int r = threadIdx.x; r < nr; r += 32) dst[r] = tile[r][kk];
    }
}

// ------------------------------------- inverse transform along z (columns)
// One snapshot: G[f][y][z][kx] = sum_kz f_hat(y, kz, kx) e^{+i kz z} for f =
// u, v, w, p, mean removed from the (0,0) coefficient.  CTA = CW adjacent kx
// columns of one (field, y) plane; dynamic shared memory (1 + 2 CW) nz complex.
template <typename TF>
__global__ void k_col_inverse(const zd* __restrict__ fields_s, int ny, int nz, int nxh, int CW,
                              const double* __restrict__ mean, const cplx<TF>* __restrict__ tw_z,
                              cplx<TF>* __restrict__ G)
{
    typedef cplx<TF> C;
    extern __shared__ __align__(16) unsigned char sh_raw_ci[];
    C* stw = (C*)sh_raw_ci;                  // [nz] twiddles
    C* b0 = stw + nz;                        // [CW][nz] x2 (ping-pong)
    C* b1 = b0 + CW * nz;
    const int kx0 = blockIdx.x * CW, y = blockIdx.y, f = blockIdx.z;
    load_twiddles(stw, tw_z, nz);
    const zd* src = fields_s + ((long long)f * ny + y) * nz * nxh;
    for (int t = threadIdx.x; t < CW * nz; t += blockDim.x) {
        int c = t % CW, kz = t / CW, kx = kx0 + c;
        zd v = mk(0.0, 0.0);
        if (kx < nxh) {
            v = src[(long long)kz * nxh + kx];
            if (kx == 0 && kz == 0) v.x -= mean[f * ny + y];
        }
        b0[c * nz + kz] = cvt<TF>(v);
    }
    const C* res = fft_block<TF, true>(b0, b1, nz, CW, nz, stw);
    C* dst = G + ((long long)f * ny + y) * nz * nxh;
    for (int t = threadIdx.x; t < CW * nz; t += blockDim.x) {
        int c = t % CW, z = t / CW, kx = kx0 + c;
        if (kx < nxh) dst[(long long)z * nxh + kx] = res[c * nz + z];
    }
}

// Register-FFT versions of the column passes for nz = N1 N2 (two-level
// transform, fft2l): CTA = CW adjacent columns x YB planes x N2 lanes; lane n2
// of a sequence loads rows n2 + N2 m straight from global memory (consecutive
// columns = consecutive addresses), one shared-memory exchange, stores
// straight back.  The inverse pass also writes the snapshot's linear
// operands Xop[f][k][s][y] (the mean-removed coefficients, runs of YB planes)
// and flags non-finite input, so no separate loader runs.
// Shared memory: N twiddles + N1 (N2 CW YB + 1) complex.
template <typename TF, int N1, int N2>
__global__ void __launch_bounds__(512)
k_col_inverse_r(const zd* __restrict__ fields_s, int ny, int nxh, int CW, int YB, int s, int ns,
                const double* __restrict__ mean, const cplx<TF>* __restrict__ tw_z, cplx<TF>* __restrict__ G,
                cplx<TF>* __restrict__ Xop, int* __restrict__ nonfinite)
{
    typedef cplx<TF> C;
    constexpr int N = N1 * N2;
    extern __shared__ __align__(16) unsigned char sh_raw_cir[];
    C* stw = (C*)sh_raw_cir;
    C* xs = stw + N;
    const int nseq = CW * YB;
    const int c = threadIdx.x % CW, yl = (threadIdx.x / CW) % YB, lane = threadIdx.x / nseq;
    const int kx = blockIdx.x * CW + c, y = blockIdx.y * YB + yl, f = blockIdx.z;
    const bool live = kx < nxh && y < ny;
    const long long Nk = (long long)N * nxh;
    load_twiddles(stw, tw_z, N);
    const zd* src = fields_s + ((long long)f * ny + y) * N * nxh;
    C* xop = Xop + (((long long)f * Nk + kx) * ns + s) * ny + y;
    int bad = 0;
    C v[N1];
    #pragma unroll
    for (int m = 0; m < N1; ++m) {
        const int kz = lane + N2 * m;
        zd x = mk(0.0, 0.0);
        if (live) {
            x = src[(long long)kz * nxh + kx];
            if (!isfinite(x.x) || !isfinite(x.y)) bad = 1;
            if (kx == 0 && kz == 0) x.x -= mean[f * ny + y];
            xop[(long long)kz * nxh * ns * ny] = cvt<TF>(x);
        }
        v[m] = cvt<TF>(x);
    }
    if (bad) atomicOr(nonfinite, 1);
    __syncthreads();
    fft2l<TF, N1, N2, true>(v, lane, xs + (yl * CW + c), N2 * nseq + 1, nseq, stw);
    if (live) {
        C* dst = G + ((long long)f * ny + y) * N * nxh;
        #pragma unroll
        for (int m = 0; m < N1; ++m) dst[(long long)(lane + N2 * m) * nxh + kx] = v[m];
    }
}

// forward column pass: CTA = CW columns x YB planes x N2 lanes, so that the
// operand stores (y contiguous) and the loads (kx contiguous) both come in
// runs of 32 bytes or more
template <typename TF, int N1, int N2>
__global__ void __launch_bounds__(512)
k_col_forward_r(const cplx<TF>* __restrict__ H, int ny, int nxh, int CW, int YB, int s, int ns,
                const cplx<TF>* __restrict__ tw_z, cplx<TF>* __restrict__ Xop)
{
    typedef cplx<TF> C;
    constexpr int N = N1 * N2;
    extern __shared__ __align__(16) unsigned char sh_raw_cfr[];
    C* stw = (C*)sh_raw_cfr;
    C* xs = stw + N;
    const int nseq = CW * YB;
    const int c = threadIdx.x % CW, yl = (threadIdx.x / CW) % YB, lane = threadIdx.x / nseq;
    const int kx = blockIdx.x * CW + c, y = blockIdx.y * YB + yl, j = blockIdx.z;
    const bool live = kx < nxh && y < ny;
    const int Nk = N * nxh;
    load_twiddles(stw, tw_z, N);
    const C* src = H + ((long long)j * ny + y) * N * nxh;
    C v[N1];
    #pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = live ? src[(long long)(lane + N2 * m) * nxh + kx] : mk((TF)0, (TF)0);
    __syncthreads();
    fft2l<TF, N1, N2, false>(v, lane, xs + (yl * CW + c), N2 * nseq + 1, nseq, stw);
    if (live) {
        // the pair products (uu .. vw) carry the factor 2 of the expansion
        const TF inz = (j < 6 ? (TF)2 : (TF)1) / (TF)N;
        #pragma unroll
        for (int m = 0; m < N1; ++m) {
            const long long k = (long long)(lane + N2 * m) * nxh + kx;
            Xop[((((long long)(F_UU + j)) * Nk + k) * ns + s) * ny + y] = inz * v[m];
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------ rows: C2R, products, R2C, one-point sums
// One CTA per (RZ rows, y).  Physical u, v, w, p on a row come from two
// complex inverse FFTs (u + i v, w + i p) of the Hermitian-extended half rows
// (imaginary parts at kx = 0 and kx = nx/2 dropped: plain C2R semantics).  The
// seven products uu, vv, ww, uv, uw, vw, q = u_i u_i go through four forward
// FFTs, (uu + i vv), (ww + i uv), (uw + i vw), (q + i 0), and are separated by
// the Hermitian split.  Output H[j][y][z][kx], j in product order, scaled by
// 1/nx.  Row sums of q, uv, pv, q u, q v, q w of the CTA's rows go to
// part[6][ny][gridDim.x] (reduced in a fixed order by k_reduce_partials, so
// repeated runs give bit-identical results).
// Shared memory: (1 + 8 RZ) nx complex.
template <typename TF>
__global__ void k_row_products(const cplx<TF>* __restrict__ G, int ny, int nz, int nx, int RZ,
                               const cplx<TF>* __restrict__ tw_x, cplx<TF>* __restrict__ H,
                               double* __restrict__ part)
{
    typedef cplx<TF> C;
    extern __shared__ __align__(16) unsigned char sh_raw_rp[];
    const int nxh = nx / 2 + 1;
    const int z0 = blockIdx.x * RZ, y = blockIdx.y;
    const int nrow = min(RZ, nz - z0);
    C* stw = (C*)sh_raw_rp;           // [nx] twiddles
    C* inv0 = stw + nx;               // [nrow][2][nx]  x2 (ping-pong)
    C* inv1 = inv0 + RZ * 2 * nx;
    C* fwd = inv1 + RZ * 2 * nx;      // [nrow][4][nx]; its scratch is inv0..inv1
    load_twiddles(stw, tw_x, nx);
    for (int t = threadIdx.x; t < nrow * 2 * nx; t += blockDim.x) {
        int r = t / (2 * nx), rem = t - r * 2 * nx, q = rem / nx, k = rem - q * nx;
        int z = z0 + r;
        const C* ga = G + (((long long)(2 * q) * ny + y) * nz + z) * nxh;
        const C* gb = G + (((long long)(2 * q + 1) * ny + y) * nz + z) * nxh;
        C A, B;
        if (k < nxh) { A = ga[k]; B = gb[k]; } else { A = conj(ga[nx - k]); B = conj(gb[nx - k]); }
        if (k == 0 || 2 * k == nx) { A.y = 0; B.y = 0; }
        inv0[(r * 2 + q) * nx + k] = mk(A.x - B.y, A.y + B.x);   // A + i B
    }
    const C* ph = fft_block<TF, true>(inv0, inv1, nx, 2 * nrow, nx, stw);
    double s_q = 0, s_uv = 0, s_pv = 0, s_qu = 0, s_qv = 0, s_qw = 0;
    for (int t = threadIdx.x; t < nrow * nx; t += blockDim.x) {
        int r = t / nx, x = t - r * nx;
        C a = ph[(r * 2) * nx + x], b = ph[(r * 2 + 1) * nx + x];
        TF u = a.x, v = a.y, w = b.x, p = b.y;
        TF q = u * u + v * v + w * w;
        double ud = u, vd = v, wd = w, qd = (double)ud * ud + vd * vd + wd * wd;
        s_q += qd; s_uv += ud * vd; s_pv += (double)p * vd; s_qu += qd * ud; s_qv += qd * vd; s_qw += qd * wd;
        fwd[(r * 4 + 0) * nx + x] = mk(u * u, v * v);
        fwd[(r * 4 + 1) * nx + x] = mk(w * w, u * v);
        fwd[(r * 4 + 2) * nx + x] = mk(u * w, v * w);
        fwd[(r * 4 + 3) * nx + x] = mk(q, (TF)0);
    }
    const C* sp = fft_block<TF, false>(fwd, inv0, nx, 4 * nrow, nx, stw);
    const TF inx = (TF)1 / (TF)nx;
    const TF h = (TF)0.5 * inx;
    for (int t = threadIdx.x; t < nrow * 4 * nxh; t += blockDim.x) {
        int r = t / (4 * nxh), rem = t - r * 4 * nxh, j = rem / nxh, k = rem - j * nxh;
        const C* seq = sp + (r * 4 + j) * nx;
        C Z = seq[k], Zc = conj(seq[(nx - k) % nx]);
        C A = h * (Z + Zc);
        C D = Z - Zc;
        C B = mk(h * D.y, -h * D.x);     // -i/2 (Z - Zc)
        int z = z0 + r;
        H[(((long long)(2 * j) * ny + y) * nz + z) * nxh + k] = A;
        if (j < 3) H[(((long long)(2 * j + 1) * ny + y) * nz + z) * nxh + k] = B;
    }
    // block reduction of the row sums
    __shared__ double red[6][32];
    double vals[6] = {s_q, s_uv, s_pv, s_qu, s_qv, s_qw};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = 0; i < 6; ++i) {
        double v = warp_sum(vals[i]);
        if (lane == 0) red[i][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) acc += red[threadIdx.x][w];
        part[((long long)threadIdx.x * ny + y) * gridDim.x + blockIdx.x] = acc;   // S_Q .. S_QW
    }
}

// Register-FFT row pass for nx = N1 N2 (fft2l): CTA = RZ rows x N2 lanes.
// Per row: two inverse transforms (u + i v, w + i p), the seven products in
// registers, four forward transforms, Hermitian split through shared memory.
// Row sums: FP32 over a thread's N1 points, FP64 across threads.
template <typename TF, int N1, int N2, int RZ>
__global__ void __launch_bounds__(RZ * N2)
k_row_products_r(const cplx<TF>* __restrict__ G, int ny, int nz, const cplx<TF>* __restrict__ tw_x,
                 cplx<TF>* __restrict__ H, double* __restrict__ part)
{
    typedef cplx<TF> C;
    constexpr int N = N1 * N2, nxh = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char sh_raw_rpr[];
    C* stw = (C*)sh_raw_rpr;
    C* xs = stw + N;                        // [RZ][N1][N2 + 1] exchange
    C* zb = xs + RZ * N1 * (N2 + 1);        // [RZ][4][N] forward spectra
    const int lane = threadIdx.x % N2, r = threadIdx.x / N2;
    const int z = blockIdx.x * RZ + r, y = blockIdx.y;
    const bool live = z < nz;
    const int zz = live ? z : 0;
    C* xr = xs + r * N1 * (N2 + 1);
    load_twiddles(stw, tw_x, N);
    C v0[N1], v1[N1];
    #pragma unroll
    for (int q = 0; q < 2; ++q) {
        const C* ga = G + (((long long)(2 * q) * ny + y) * nz + zz) * nxh;
        const C* gb = G + (((long long)(2 * q + 1) * ny + y) * nz + zz) * nxh;
        C* v = q ? v1 : v0;
        #pragma unroll
        for (int m = 0; m < N1; ++m) {
            const int k = lane + N2 * m;
            C A, B;
            if (k < nxh) { A = ga[k]; B = gb[k]; } else { A = conj(ga[N - k]); B = conj(gb[N - k]); }
            if (k == 0 || 2 * k == N) { A.y = 0; B.y = 0; }
            v[m] = mk(A.x - B.y, A.y + B.x);     // A + i B
        }
        __syncthreads();
        fft2l<TF, N1, N2, true>(v, lane, xr, N2 + 1, 1, stw);
    }
    // v0[m] = u + i v, v1[m] = w + i p at x = lane + N2 m
    TF s6[6] = {0, 0, 0, 0, 0, 0};
    #pragma unroll
    for (int m = 0; m < N1; ++m) {
        const TF u = v0[m].x, vv = v0[m].y, w = v1[m].x, pp = v1[m].y;
        const TF q = u * u + vv * vv + w * w;
        s6[0] += q; s6[1] += u * vv; s6[2] += pp * vv; s6[3] += q * u; s6[4] += q * vv; s6[5] += q * w;
    }
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
        C f[N1];
        #pragma unroll
        for (int m = 0; m < N1; ++m) {
            const TF u = v0[m].x, vv = v0[m].y, w = v1[m].x;
            if (j == 0) f[m] = mk(u * u, vv * vv);
            else if (j == 1) f[m] = mk(w * w, u * vv);
            else if (j == 2) f[m] = mk(u * w, vv * w);
            else f[m] = mk(u * u + vv * vv + w * w, (TF)0);
        }
        __syncthreads();
        fft2l<TF, N1, N2, false>(f, lane, xr, N2 + 1, 1, stw);
        #pragma unroll
        for (int m = 0; m < N1; ++m) zb[(r * 4 + j) * N + lane + N2 * m] = f[m];
    }
    __syncthreads();
    const TF h = (TF)0.5 / (TF)N;
    if (live) {
        for (int it = lane; it < 4 * nxh; it += N2) {
            const int j = it / nxh, k = it - j * nxh;
            const C* seq = zb + (r * 4 + j) * N;
            const C Z = seq[k], Zc = conj(seq[(N - k) & (N - 1)]);
            const C A = h * (Z + Zc);
            const C D = Z - Zc;
            const C B = mk(h * D.y, -h * D.x);     // -i/2 (Z - Zc)
            H[(((long long)(2 * j) * ny + y) * nz + z) * nxh + k] = A;
            if (j < 3) H[(((long long)(2 * j + 1) * ny + y) * nz + z) * nxh + k] = B;
        }
    }
    // block reduction of the row sums (FP64 across threads)
    __shared__ double red[6][32];
    const int wl = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = 0; i < 6; ++i) {
        double v = live ? (double)s6[i] : 0.0;
        v = warp_sum(v);
        if (wl == 0) red[i][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) acc += red[threadIdx.x][w];
        part[((long long)threadIdx.x * ny + y) * gridDim.x + blockIdx.x] = acc;
    }
}

// ---------------------------------- forward transform along z (columns)
// One snapshot: Xop[4 + j][k][s][y] = (c_j/nz) sum_z H[j][y][z][kx] e^{-i kz z}
// for the seven products, c_j = 2 for the pair products uu .. vw (the factor
// 2 of the correlation expansion, Eq. 7) and 1 for q.  CTA = CW kx columns x YB planes of one product;
// dynamic shared memory (1 + 2 CW YB) nz complex.
template <typename TF>
__global__ void k_col_forward(const cplx<TF>* __restrict__ H, int ny, int nz, int nxh, int CW, int YB,
                              int s, int ns, const cplx<TF>* __restrict__ tw_z, cplx<TF>* __restrict__ Xop)
{
    typedef cplx<TF> C;
    extern __shared__ __align__(16) unsigned char sh_raw_cf[];
    C* stw = (C*)sh_raw_cf;                 // [nz] twiddles
    const int nb = CW * YB;
    C* b0 = stw + nz;                       // [nb][nz] x2 (ping-pong)
    C* b1 = b0 + nb * nz;
    const int kx0 = blockIdx.x * CW, y0 = blockIdx.y * YB, j = blockIdx.z;
    const int Nk = nz * nxh;
    load_twiddles(stw, tw_z, nz);
    for (int t = threadIdx.x; t < nb * nz; t += blockDim.x) {
        int c = t % CW, rem = t / CW, yy = rem % YB, z = rem / YB;
        int kx = kx0 + c, y = y0 + yy;
        C v = mk((TF)0, (TF)0);
        if (kx < nxh && y < ny) v = H[(((long long)j * ny + y) * nz + z) * nxh + kx];
        b0[(yy * CW + c) * nz + z] = v;
    }
    const C* res = fft_block<TF, false>(b0, b1, nz, nb, nz, stw);
    const TF inz = (j < 6 ? (TF)2 : (TF)1) / (TF)nz;     // pair products carry the factor 2 of the expansion
    for (int t = threadIdx.x; t < nb * nz; t += blockDim.x) {
        int yy = t % YB, rem = t / YB, c = rem % CW, kz = rem / CW;
        int kx = kx0 + c, y = y0 + yy;
        if (kx < nxh && y < ny) {
            long long k = (long long)kz * nxh + kx;
            Xop[((((long long)(F_UU + j)) * Nk + k) * ns + s) * ny + y] = inz * res[(yy * CW + c) * nz + kz];
        }
    }
}

// ------------------------------------------------- pseudo-dissipation
// Parseval form of <d_j u_i d_j u_i> (Sec. 2): for one chunk of wavenumbers,
//   part[y][chunk] = sum_{s, k in chunk, i} w_k [ (kx^2 + kz^2) |u_i(y,k)|^2 + |d_y u_i(y,k)|^2 ],
// d_y by the 5-point FD stencil applied to the coefficients (it commutes with
// the transform); w_k = 1 on the kx = 0 and kx = nx/2 lines, 2 elsewhere (half
// spectrum).  One thread per y; arithmetic in TF, the running sum compensated
// (Kahan) so an FP32 pass keeps ~1e-7 relative accuracy; partials reduced in
// FP64 in a fixed order by k_reduce_partials.
template <typename TF>
__global__ void k_eps(const cplx<TF>* __restrict__ Xop, int ns, int ny, int nz, int nxh, int nx,
                      double Lx, double Lz, const double* __restrict__ fdw, const int* __restrict__ fdl0,
                      int kchunk, double* __restrict__ part)
{
    const int Nk = nz * nxh;
    const int kbeg = blockIdx.x * kchunk, kend = min(Nk, kbeg + kchunk);
    const TF cx = (TF)(2.0 * 3.14159265358979323846 / Lx), cz = (TF)(2.0 * 3.14159265358979323846 / Lz);
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
        const int l0 = fdl0[y];
        TF w5[5];
        for (int l = 0; l < 5; ++l) w5[l] = (TF)fdw[5 * y + l];
        TF sum = 0, comp = 0;
        for (int k = kbeg; k < kend; ++k) {
            const int kz_i = k / nxh, kx_i = k - kz_i * nxh;
            const TF kx = cx * (TF)signed_bin(kx_i, nx), kz = cz * (TF)signed_bin(kz_i, nz);
            const TF wk = (kx_i == 0 || 2 * kx_i == nx) ? (TF)1 : (TF)2;
            const TF k2 = kx * kx + kz * kz;
            TF acc = 0;
            for (int i = 0; i < 3; ++i)
                for (int s = 0; s < ns; ++s) {
                    const cplx<TF>* col = Xop + (((long long)i * Nk + k) * ns + s) * ny;
                    const cplx<TF> a = col[y];
                    TF dr = 0, di = 0;
                    #pragma unroll
                    for (int l = 0; l < 5; ++l) { const cplx<TF> b = col[l0 + l]; dr += w5[l] * b.x; di += w5[l] * b.y; }
                    acc += k2 * (a.x * a.x + a.y * a.y) + dr * dr + di * di;
                }
            // compensated add of this wavenumber's contribution
            const TF yk = wk * acc - comp;
            const TF t = sum + yk;
            comp = (t - sum) - yk;
            sum = t;
        }
        part[(long long)y * gridDim.x + blockIdx.x] = (double)sum;
    }
}

// out[j] += sum_b part[j * nb + b], b in increasing order (deterministic)
__global__ void k_reduce_partials(const double* __restrict__ part, int nvals, int nb, double* __restrict__ out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nvals) return;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += part[(long long)j * nb + b];
    out[j] += acc;
}

// ------------------------------------------------------------------ host
// Launch sequence of the products stage for one batch (snapshots one by one).
template <typename TF>
int products_launch(const ProdArgs& a)
{
    typedef cplx<TF> C;
    const int ny = a.ny, Nk = a.Nk, nxh = a.nxh, nz = a.nz, nx = a.nx, ns = a.ns;
    cudaStream_t st = a.st;
    C* Xop = (C*)a.Xop;
    int launches = 0;
    const int nch = (ny + ll_rows<TF>() - 1) / ll_rows<TF>(), rows = (ny + nch - 1) / nch;
    // at nz = 256 the register column pass writes the linear operands itself
    const bool fused_load = nz == 256;
    if (!a.up_ev && !fused_load) {
        k_load_linear<TF><<<dim3((Nk + 31) / 32, nch, ns * 4), dim3(32, 8), 0, st>>>(a.fields, ns, ny, Nk, rows, 0,
                                                                                      a.mean, Xop, a.nonfinite);
        ++launches;
    }
    // With a second stream and second G, H, part buffers, snapshot s runs on
    // stream s % 2, so the transforms of two snapshots overlap; the row sums
    // are still reduced into stats on the main stream in snapshot order.
    const bool two = a.st2 != nullptr && a.G2 != nullptr && a.H2 != nullptr && a.part2 != nullptr;
    cudaEvent_t ev_start = nullptr, ev_rp[2] = {nullptr, nullptr}, ev_red[2] = {nullptr, nullptr},
                ev_end = nullptr;
    if (two) {
        if (a.ev) {
            ev_start = a.ev[0]; ev_end = a.ev[1];
            ev_rp[0] = a.ev[2]; ev_rp[1] = a.ev[3]; ev_red[0] = a.ev[4]; ev_red[1] = a.ev[5];
        } else {
            cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
            cudaEventCreateWithFlags(&ev_end, cudaEventDisableTiming);
            for (int i = 0; i < 2; ++i) {
                cudaEventCreateWithFlags(&ev_rp[i], cudaEventDisableTiming);
                cudaEventCreateWithFlags(&ev_red[i], cudaEventDisableTiming);
            }
        }
        cudaEventRecord(ev_start, st);                   // the second stream starts after earlier work
        cudaStreamWaitEvent(a.st2, ev_start, 0);
    }
    for (int s = 0; s < ns; ++s) {
        const zd* fs = a.fields + (size_t)s * 4 * ny * Nk;
        const int b = two ? (s & 1) : 0;
        cudaStream_t ss = b ? a.st2 : st;
        C* G = (C*)(b ? a.G2 : a.G);
        C* H = (C*)(b ? a.H2 : a.H);
        double* part = b ? a.part2 : a.part;
        if (two && s >= 2) cudaStreamWaitEvent(ss, ev_red[b], 0);     // part[b] read by the last reduction
        if (a.up_ev) cudaStreamWaitEvent(ss, a.up_ev[s], 0);    // this snapshot's data arrive on the upload stream
        if (a.up_ev && !fused_load) {
            k_load_linear<TF><<<dim3((Nk + 31) / 32, nch, 4), dim3(32, 8), 0, ss>>>(a.fields, ns, ny, Nk, rows, s,
                                                                                     a.mean, Xop, a.nonfinite);
            ++launches;
        }
        if (nz == 256) {
            // FP32: 4 kx x 8 planes per CTA; FP64 4 x 4 (shared memory)
            constexpr int CWR = 4, YBR = sizeof(TF) == 4 ? 8 : 4;
            k_col_inverse_r<TF, 16, 16><<<dim3((nxh + CWR - 1) / CWR, (ny + YBR - 1) / YBR, 4), CWR * YBR * 16,
                                          (256 + 16 * (16 * CWR * YBR + 1)) * sizeof(C), ss>>>(
                fs, ny, nxh, CWR, YBR, s, ns, a.mean, (const C*)a.tw_z, G, Xop, a.nonfinite);
        } else {
            k_col_inverse<TF><<<dim3((nxh + a.cw_ci - 1) / a.cw_ci, ny, 4), 256, (1 + 2 * a.cw_ci) * nz * sizeof(C), ss>>>(
                fs, ny, nz, nxh, a.cw_ci, a.mean, (const C*)a.tw_z, G);
        }
        const int nrb = (nx == 256) ? (nz + 3) / 4 : (nz + a.rz_rp - 1) / a.rz_rp;
        if (nx == 256) {
            k_row_products_r<TF, 16, 16, 4><<<dim3(nrb, ny), 4 * 16, (256 + 4 * 16 * 17 + 4 * 4 * 256) * sizeof(C),
                                              ss>>>((const C*)G, ny, nz, (const C*)a.tw_x, H, part);
        } else {
            k_row_products<TF><<<dim3(nrb, ny), 256, (1 + 8 * a.rz_rp) * nx * sizeof(C), ss>>>(
                (const C*)G, ny, nz, nx, a.rz_rp, (const C*)a.tw_x, H, part);
        }
        if (two) {
            cudaEventRecord(ev_rp[b], ss);
            cudaStreamWaitEvent(st, ev_rp[b], 0);
        }
        k_reduce_partials<<<(6 * ny + 127) / 128, 128, 0, st>>>(part, 6 * ny, nrb, a.stats);
        if (two) cudaEventRecord(ev_red[b], st);
        if (nz == 256) {
            // FP32: 8 planes per CTA (the operand stores come in 64-byte runs);
            // FP64 keeps 4 (its exchange buffer would hold one CTA per SM)
            constexpr int CWR = 4, YBR = sizeof(TF) == 4 ? 8 : 4;
            k_col_forward_r<TF, 16, 16><<<dim3((nxh + CWR - 1) / CWR, (ny + YBR - 1) / YBR, 7), CWR * YBR * 16,
                                          (256 + 16 * (16 * CWR * YBR + 1)) * sizeof(C), ss>>>(
                (const C*)H, ny, nxh, CWR, YBR, s, ns, (const C*)a.tw_z, Xop);
        } else {
            k_col_forward<TF><<<dim3((nxh + a.cw_cf - 1) / a.cw_cf, (ny + a.yb_cf - 1) / a.yb_cf, 7), 256,
                                (1 + 2 * a.cw_cf * a.yb_cf) * nz * sizeof(C), ss>>>(
                (const C*)H, ny, nz, nxh, a.cw_cf, a.yb_cf, s, ns, (const C*)a.tw_z, Xop);
        }
        launches += 4;
    }
    if (two) {
        // join: the main stream waits for the second stream's last transforms
        cudaEventRecord(ev_end, a.st2);
        cudaStreamWaitEvent(st, ev_end, 0);
        if (!a.ev) {
            cudaEventDestroy(ev_start);
            cudaEventDestroy(ev_end);
            for (int i = 0; i < 2; ++i) {
                cudaEventDestroy(ev_rp[i]);
                cudaEventDestroy(ev_red[i]);
            }
        }
    }
    const int neb = (Nk + a.eps_kchunk - 1) / a.eps_kchunk;
    // one thread per wall-normal row: no second pass for a ragged last row
    const int eps_threads = std::min(1024, (ny + 31) / 32 * 32);
    k_eps<TF><<<neb, eps_threads, 0, st>>>(Xop, ns, ny, nz, nxh, nx, a.Lx, a.Lz, a.fdw, a.fdl0, a.eps_kchunk,
                                          a.part);
    k_reduce_partials<<<(ny + 127) / 128, 128, 0, st>>>(a.part, ny, neb, a.stats + S_EPS * ny);
    return launches + 2;
}
template int products_launch<double>(const ProdArgs&);
template int products_launch<float>(const ProdArgs&);

static cudaError_t set_dyn_smem(const void* k, int lim)
{
    cudaFuncAttributes fa;
    cudaError_t r = cudaFuncGetAttributes(&fa, k);
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - (int)fa.sharedSizeBytes);
    return r;
}

cudaError_t products_set_attrs(int lim)
{
    const void* ks[] = {(const void*)k_col_inverse<double>, (const void*)k_row_products<double>,
                        (const void*)k_col_forward<double>, (const void*)k_col_inverse<float>,
                        (const void*)k_row_products<float>, (const void*)k_col_forward<float>,
                        (const void*)k_col_inverse_r<double, 16, 16>, (const void*)k_col_inverse_r<float, 16, 16>,
                        (const void*)k_col_forward_r<double, 16, 16>, (const void*)k_col_forward_r<float, 16, 16>,
                        (const void*)k_row_products_r<double, 16, 16, 4>, (const void*)k_row_products_r<float, 16, 16, 4>};
    cudaError_t e = cudaSuccess;
    for (const void* k : ks) { cudaError_t r = set_dyn_smem(k, lim); if (r != cudaSuccess) e = r; }
    return e;
}

// explicit instantiations
#define GKE_INST(TF)                                                                                       \
    template __global__ void k_load_linear<TF>(const zd*, int, int, int, int, int, const double*, cplx<TF>*,   \
                                               int*);                                                        \
    template __global__ void k_col_inverse<TF>(const zd*, int, int, int, int, const double*,               \
                                               const cplx<TF>*, cplx<TF>*);                                \
    template __global__ void k_row_products<TF>(const cplx<TF>*, int, int, int, int, const cplx<TF>*,      \
                                                cplx<TF>*, double*);                                       \
    template __global__ void k_col_forward<TF>(const cplx<TF>*, int, int, int, int, int, int, int,         \
                                               const cplx<TF>*, cplx<TF>*);                                \
    template __global__ void k_eps<TF>(const cplx<TF>*, int, int, int, int, int, double, double,           \
                                       const double*, const int*, int, double*);
GKE_INST(double)
GKE_INST(float)
#undef GKE_INST

}  // namespace gke
