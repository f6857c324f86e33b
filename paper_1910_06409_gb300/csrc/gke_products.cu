// gke_products.cu -- Step 1 (ensemble mean) and the per-snapshot part of
// Step 2 that precedes the correlations: fluctuations, the in-plane products
// formed in physical space (Sec. 3.1: widehat{uu} = F(u u)), their forward
// transforms, and the one-point statistics the assembly needs.
//
// Transforms along z act on tiles of adjacent kx columns; transforms along x
// on two real rows at a time (packed as real and imaginary part of one
// complex sequence).  All in FP64.
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

// ---------------------------------------------- linear fields -> operands
// Xop[f][k][s][y] = fields[s][f][y][k] - mean_f(y) [k == 0], f = u, v, w, p.
// 32x32 (k, y) tile transpose through shared memory; flags non-finite input.
__global__ void k_load_linear(const zd* __restrict__ fields, int ns, int ny, int Nk,
                              const double* __restrict__ mean, zd* __restrict__ Xop,
                              int* __restrict__ nonfinite)
{
    __shared__ zd tile[32][33];
    const int k0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int s = blockIdx.z / 4, f = blockIdx.z % 4;
    int bad = 0;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int y = y0 + r, k = k0 + threadIdx.x;
        if (y < ny && k < Nk) {
            zd v = fields[(((long long)s * 4 + f) * ny + y) * Nk + k];
            if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
            if (k == 0) v.x -= mean[f * ny + y];
            tile[r][threadIdx.x] = v;
        }
    }
    if (bad) atomicOr(nonfinite, 1);
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int k = k0 + r, y = y0 + threadIdx.x;
        if (y < ny && k < Nk) Xop[(((long long)f * Nk + k) * ns + s) * ny + y] = tile[threadIdx.x][r];
    }
}

// ------------------------------------- inverse transform along z (columns)
// One snapshot: G[f][y][z][kx] = sum_kz f_hat(y, kz, kx) e^{+i kz z} for f =
// u, v, w, p, mean removed from the (0,0) coefficient.  CTA = CW adjacent kx
// columns of one (field, y) plane; dynamic shared memory CW * nz complex.
__global__ void k_col_inverse(const zd* __restrict__ fields_s, int ny, int nz, int nxh, int CW,
                              const double* __restrict__ mean, const zd* __restrict__ tw_z,
                              zd* __restrict__ G)
{
    extern __shared__ zd sh_ci[];
    const int kx0 = blockIdx.x * CW, y = blockIdx.y, f = blockIdx.z;
    const int lg = ilog2(nz);
    const zd* src = fields_s + ((long long)f * ny + y) * nz * nxh;
    for (int t = threadIdx.x; t < CW * nz; t += blockDim.x) {
        int c = t % CW, kz = t / CW, kx = kx0 + c;
        zd v = mk(0.0, 0.0);
        if (kx < nxh) {
            v = src[(long long)kz * nxh + kx];
            if (kx == 0 && kz == 0) v.x -= mean[f * ny + y];
        }
        sh_ci[c * nz + bitrev(kz, lg)] = v;
    }
    fft_radix2_block(sh_ci, nz, CW, lg, tw_z, +1);
    zd* dst = G + ((long long)f * ny + y) * nz * nxh;
    for (int t = threadIdx.x; t < CW * nz; t += blockDim.x) {
        int c = t % CW, z = t / CW, kx = kx0 + c;
        if (kx < nxh) dst[(long long)z * nxh + kx] = sh_ci[c * nz + z];
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
// Shared memory: RZ * 6 * nx complex.
__global__ void k_row_products(const zd* __restrict__ G, int ny, int nz, int nx, int RZ,
                               const zd* __restrict__ tw_x, zd* __restrict__ H,
                               double* __restrict__ part)
{
    extern __shared__ zd sh_rp[];
    const int nxh = nx / 2 + 1, lg = ilog2(nx);
    const int z0 = blockIdx.x * RZ, y = blockIdx.y;
    const int nrow = min(RZ, nz - z0);
    zd* inv = sh_rp;                  // [nrow][2][nx]
    zd* fwd = sh_rp + RZ * 2 * nx;    // [nrow][4][nx]
    for (int t = threadIdx.x; t < nrow * 2 * nx; t += blockDim.x) {
        int r = t / (2 * nx), rem = t - r * 2 * nx, q = rem / nx, k = rem - q * nx;
        int z = z0 + r;
        const zd* ga = G + (((long long)(2 * q) * ny + y) * nz + z) * nxh;
        const zd* gb = G + (((long long)(2 * q + 1) * ny + y) * nz + z) * nxh;
        zd A, B;
        if (k < nxh) { A = ga[k]; B = gb[k]; } else { A = conj(ga[nx - k]); B = conj(gb[nx - k]); }
        if (k == 0 || 2 * k == nx) { A.y = 0.0; B.y = 0.0; }
        inv[(r * 2 + q) * nx + bitrev(k, lg)] = mk(A.x - B.y, A.y + B.x);   // A + i B
    }
    fft_radix2_block(inv, nx, 2 * nrow, lg, tw_x, +1);
    double s_q = 0, s_uv = 0, s_pv = 0, s_qu = 0, s_qv = 0, s_qw = 0;
    for (int t = threadIdx.x; t < nrow * nx; t += blockDim.x) {
        int r = t / nx, x = t - r * nx;
        zd a = inv[(r * 2) * nx + x], b = inv[(r * 2 + 1) * nx + x];
        double u = a.x, v = a.y, w = b.x, p = b.y;
        double q = u * u + v * v + w * w;
        s_q += q; s_uv += u * v; s_pv += p * v; s_qu += q * u; s_qv += q * v; s_qw += q * w;
        int br = bitrev(x, lg);
        fwd[(r * 4 + 0) * nx + br] = mk(u * u, v * v);
        fwd[(r * 4 + 1) * nx + br] = mk(w * w, u * v);
        fwd[(r * 4 + 2) * nx + br] = mk(u * w, v * w);
        fwd[(r * 4 + 3) * nx + br] = mk(q, 0.0);
    }
    fft_radix2_block(fwd, nx, 4 * nrow, lg, tw_x, -1);
    const double inx = 1.0 / nx;
    for (int t = threadIdx.x; t < nrow * 4 * nxh; t += blockDim.x) {
        int r = t / (4 * nxh), rem = t - r * 4 * nxh, j = rem / nxh, k = rem - j * nxh;
        const zd* seq = fwd + (r * 4 + j) * nx;
        zd Z = seq[k], Zc = conj(seq[(nx - k) & (nx - 1)]);
        zd A = (0.5 * inx) * (Z + Zc);
        zd D = Z - Zc;
        zd B = mk(0.5 * inx * D.y, -0.5 * inx * D.x);     // -i/2 (Z - Zc)
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

// ---------------------------------- forward transform along z (columns)
// One snapshot: Xop[4 + j][k][s][y] = (1/nz) sum_z H[j][y][z][kx] e^{-i kz z}
// for the seven products.  CTA = CW kx columns x YB planes of one product;
// dynamic shared memory CW * YB * nz complex.
__global__ void k_col_forward(const zd* __restrict__ H, int ny, int nz, int nxh, int CW, int YB,
                              int s, int ns, const zd* __restrict__ tw_z, zd* __restrict__ Xop)
{
    extern __shared__ zd sh_cf[];
    const int kx0 = blockIdx.x * CW, y0 = blockIdx.y * YB, j = blockIdx.z;
    const int lg = ilog2(nz);
    const int Nk = nz * nxh;
    const int nb = CW * YB;
    for (int t = threadIdx.x; t < nb * nz; t += blockDim.x) {
        int c = t % CW, rem = t / CW, yy = rem % YB, z = rem / YB;
        int kx = kx0 + c, y = y0 + yy;
        zd v = mk(0.0, 0.0);
        if (kx < nxh && y < ny) v = H[(((long long)j * ny + y) * nz + z) * nxh + kx];
        sh_cf[(yy * CW + c) * nz + bitrev(z, lg)] = v;
    }
    fft_radix2_block(sh_cf, nz, nb, lg, tw_z, -1);
    const double inz = 1.0 / nz;
    for (int t = threadIdx.x; t < nb * nz; t += blockDim.x) {
        int yy = t % YB, rem = t / YB, c = rem % CW, kz = rem / CW;
        int kx = kx0 + c, y = y0 + yy;
        if (kx < nxh && y < ny) {
            long long k = (long long)kz * nxh + kx;
            Xop[((((long long)(F_UU + j)) * Nk + k) * ns + s) * ny + y] = inz * sh_cf[(yy * CW + c) * nz + kz];
        }
    }
}

// ------------------------------------------------- pseudo-dissipation
// Parseval form of <d_j u_i d_j u_i> (Sec. 2): for one chunk of wavenumbers,
//   part[y][chunk] = sum_{s, k in chunk, i} w_k [ (kx^2 + kz^2) |u_i(y,k)|^2 + |d_y u_i(y,k)|^2 ],
// d_y by the 5-point FD stencil applied to the coefficients (it commutes with
// the transform); w_k = 1 on the kx = 0 and kx = nx/2 lines, 2 elsewhere (half
// spectrum).  One thread per y; partials reduced in a fixed order later.
__global__ void k_eps(const zd* __restrict__ Xop, int ns, int ny, int nz, int nxh, int nx,
                      double Lx, double Lz, const double* __restrict__ fdw, const int* __restrict__ fdl0,
                      int kchunk, double* __restrict__ part)
{
    const int Nk = nz * nxh;
    const int kbeg = blockIdx.x * kchunk, kend = min(Nk, kbeg + kchunk);
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
        const int l0 = fdl0[y];
        double w5[5];
        for (int l = 0; l < 5; ++l) w5[l] = fdw[5 * y + l];
        double acc = 0.0;
        for (int k = kbeg; k < kend; ++k) {
            int kz_i = k / nxh, kx_i = k - kz_i * nxh;
            double kx = 2.0 * 3.14159265358979323846 * signed_bin(kx_i, nx) / Lx;
            double kz = 2.0 * 3.14159265358979323846 * signed_bin(kz_i, nz) / Lz;
            double wk = (kx_i == 0 || 2 * kx_i == nx) ? 1.0 : 2.0;
            double k2 = kx * kx + kz * kz;
            for (int i = 0; i < 3; ++i)
                for (int s = 0; s < ns; ++s) {
                    const zd* col = Xop + (((long long)i * Nk + k) * ns + s) * ny;
                    zd a = col[y];
                    zd d = mk(0.0, 0.0);
                    for (int l = 0; l < 5; ++l) d = d + w5[l] * col[l0 + l];
                    acc += wk * (k2 * (a.x * a.x + a.y * a.y) + d.x * d.x + d.y * d.y);
                }
        }
        part[(long long)y * gridDim.x + blockIdx.x] = acc;
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

}  // namespace gke
