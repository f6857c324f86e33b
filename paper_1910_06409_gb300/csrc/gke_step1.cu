// gke_step1.cu -- Step 1 for velocity-vorticity databases (Sec. 3.2, Step 1).
//
// DNS solvers in velocity-vorticity form store the wall-normal velocity v and
// vorticity eta = du/dz - dw/dx as Fourier coefficients in x, z, plus the plane
// averages of u and w.  Step 1 recovers u, w and the pressure p per snapshot,
// all in FP64, as the fields [4][ny][nz][nxh] the GKE path consumes:
//   k_s1_velocity     u = (i kx dv/dy - i kz eta) / k^2, w = (i kz dv/dy + i kx eta) / k^2
//                     (continuity and the definition of eta solved for u, w);
//   k_s1_col          inverse / forward DFT along z of column groups (fft_block);
//   k_s1_row_products per (y, z) row: inverse real DFT along x of u, v, w
//                     (u + i v and w as complex sequences), the six products
//                     u_i u_j, forward DFT of them packed in pairs;
//   k_s1_factor       LU (partial pivoting) of the banded Poisson operator
//                     d2/dy2 - k^2 with its Neumann wall rows, once per plan;
//   k_s1_poisson      the source -d_i d_j (u_i u_j) and the wall values
//                     dp/dy = nu d2v/dy2 (y-momentum at no-slip walls), then
//                     the banded solve, per wavenumber.
// Conventions: odd x / z derivatives use the signed wavenumber with 0 on the
// Nyquist lines, second derivatives the true square; d/dy and d2/dy2 are the
// 5-point weights on the nodes l0 .. l0 + 4 of each row; the singular (0, 0)
// Poisson problem has its first row replaced by p(y_0) = 0.
#include "gke_common.cuh"
#include "gke_kernels.h"

namespace gke {

// band of the Poisson rows: interior rows reach 2 below and 2 above the
// diagonal, the one-sided wall rows 4; partial pivoting adds S1_KL columns
// of fill above, so a row is stored from col r - KL to r + KU + KL
constexpr int S1_KL = 4, S1_KU = 4, S1_W = 2 * S1_KL + S1_KU + 1;
constexpr double TWO_PI = 6.283185307179586476925286766559;

__device__ __forceinline__ double kodd(int m, int n, double L) { return TWO_PI * signed_bin(m, n) / L; }
__device__ __forceinline__ double ktrue2(int m, int n, double L)
{
    const int s = (2 * m > n) ? m - n : m;           // the true bin on the Nyquist line
    const double k = TWO_PI * s / L;
    return k * k;
}

// u, w of one snapshot; v copied; (0, 0) modes from the plane averages
__global__ void k_s1_velocity(const zd* __restrict__ v, const zd* __restrict__ eta, const double* __restrict__ mean_uw,
                              int ny, int nz, int nx, double Lx, double Lz, const double* __restrict__ w1,
                              const int* __restrict__ l0, zd* __restrict__ out)
{
    const int nxh = nx / 2 + 1;
    const long long Nk = (long long)nz * nxh;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)ny * Nk) return;
    const int j = (int)(i / Nk);
    const long long k = i - j * Nk;
    const int kz_i = (int)(k / nxh), kx_i = (int)(k - (long long)kz_i * nxh);
    const double kx = kodd(kx_i, nx, Lx), kz = kodd(kz_i, nz, Lz), k2 = kx * kx + kz * kz;
    zd dv = mk(0.0, 0.0);
    for (int l = 0; l < 5; ++l) {
        const zd a = v[(long long)(l0[j] + l) * Nk + k];
        dv = mk(dv.x + w1[5 * j + l] * a.x, dv.y + w1[5 * j + l] * a.y);
    }
    const zd e = eta[i];
    zd u = mk(0.0, 0.0), w = u;
    if (k == 0) {
        u = mk(mean_uw[j], 0.0);
        w = mk(mean_uw[ny + j], 0.0);
    } else if (k2 > 0.0) {
        // i kx dv - i kz e, i kz dv + i kx e, over k^2
        u = mk((-kx * dv.y + kz * e.y) / k2, (kx * dv.x - kz * e.x) / k2);
        w = mk((-kz * dv.y - kx * e.y) / k2, (kz * dv.x + kx * e.x) / k2);
    }
    const long long fs = (long long)ny * Nk;
    out[i] = u;
    out[fs + i] = v[i];
    out[2 * fs + i] = w;
}

// DFT along z of nf fields [f][ny][nz][nxh]: CTA = (field, y, NC columns kx);
// INV: unnormalised inverse; forward: scaled by 1 / nz
template <bool INV>
__global__ void k_s1_col(const zd* __restrict__ in, int ny, int nz, int nxh, int NC, const zd* __restrict__ tw,
                         zd* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char sh_s1c[];
    zd* stw = (zd*)sh_s1c;
    zd* xa = stw + nz;
    zd* xb = xa + (size_t)NC * nz;
    const int f = blockIdx.z, j = blockIdx.y, kx0 = blockIdx.x * NC;
    const long long plane = ((long long)f * ny + j) * nz * nxh;
    load_twiddles(stw, tw, nz);
    for (int e = threadIdx.x; e < NC * nz; e += blockDim.x) {
        const int c = e % NC, kz = e / NC;
        xa[(size_t)c * nz + kz] = (kx0 + c < nxh) ? in[plane + (long long)kz * nxh + kx0 + c] : mk(0.0, 0.0);
    }
    const zd* r = fft_block<double, INV>(xa, xb, nz, NC, nz, stw);
    const double sc = INV ? 1.0 : 1.0 / nz;
    for (int e = threadIdx.x; e < NC * nz; e += blockDim.x) {
        const int c = e % NC, z = e / NC;
        if (kx0 + c < nxh) {
            const zd a = r[(size_t)c * nz + z];
            out[plane + (long long)z * nxh + kx0 + c] = mk(sc * a.x, sc * a.y);
        }
    }
}

// One (y, z) row: A[3][ny][nz][nxh] (x half spectra of u, v, w at fixed z)
// -> the x half spectra of uu, uv, uw, vv, vw, ww, scaled by 1 / nx, into
// B[6][ny][nz][nxh].
__global__ void k_s1_row_products(const zd* __restrict__ A, int ny, int nz, int nx, const zd* __restrict__ tw,
                                  zd* __restrict__ B)
{
    extern __shared__ __align__(16) unsigned char sh_s1r[];
    const int nxh = nx / 2 + 1;
    zd* stw = (zd*)sh_s1r;
    zd* xa = stw + nx;                 // 3 sequences of nx
    zd* xb = xa + 3 * (size_t)nx;      // 3 sequences of nx
    const int z = blockIdx.x, j = blockIdx.y;
    const long long fs = (long long)ny * nz * nxh, row = ((long long)j * nz + z) * nxh;
    load_twiddles(stw, tw, nx);
    // Hermitian extension of a half spectrum; the kx = 0 and nx/2 bins keep
    // their real parts (a real sequence's DFT is real there)
    auto H = [&](int f, int m) -> zd {
        if (m == 0 || 2 * m == nx) return mk(A[f * fs + row + m].x, 0.0);
        if (2 * m < nx) return A[f * fs + row + m];
        const zd a = A[f * fs + row + (nx - m)];
        return mk(a.x, -a.y);
    };
    for (int m = threadIdx.x; m < nx; m += blockDim.x) {
        const zd u = H(0, m), v = H(1, m), w = H(2, m);
        xa[m] = mk(u.x - v.y, u.y + v.x);             // U + i V
        xa[nx + m] = w;
    }
    zd* r = fft_block<double, true>(xa, xb, nx, 2, nx, stw);    // u + i v, w (+ 0 i)
    zd* o = (r == xa) ? xb : xa;
    for (int m = threadIdx.x; m < nx; m += blockDim.x) {
        const double u = r[m].x, v = r[m].y, w = r[nx + m].x;
        o[m] = mk(u * u, v * v);                        // uu + i vv
        o[nx + m] = mk(w * w, u * v);                   // ww + i uv
        o[2 * nx + m] = mk(u * w, v * w);               // uw + i vw
    }
    zd* q = fft_block<double, false>(o, r, nx, 3, nx, stw);
    // unpack a + i b: a^(m) = (Z(m) + conj Z(-m)) / 2, b^(m) = (Z(m) - conj Z(-m)) / (2 i)
    const double sc = 0.5 / nx;
    // output product index of (sequence, part): uu 0, uv 1, uw 2, vv 3, vw 4, ww 5
    const int dst[3][2] = {{0, 3}, {5, 1}, {2, 4}};
    for (int e = threadIdx.x; e < 3 * nxh; e += blockDim.x) {
        const int s = e / nxh, m = e - s * nxh;
        const zd Z = q[(size_t)s * nx + m], Zc = q[(size_t)s * nx + (nx - m) % nx];
        B[dst[s][0] * fs + row + m] = mk(sc * (Z.x + Zc.x), sc * (Z.y - Zc.y));
        B[dst[s][1] * fs + row + m] = mk(sc * (Z.y + Zc.y), sc * (Zc.x - Z.x));
    }
}

// band storage of wavenumber k: row r, column c (|c - r| within the window)
__device__ __forceinline__ double& band(double* ab, long long Nk, long long k, int r, int c)
{
    return ab[((long long)r * S1_W + (c - r + S1_KL)) * Nk + k];
}

// LU with partial pivoting of the Poisson operator of every wavenumber
__global__ void k_s1_factor(int ny, int nz, int nx, double Lx, double Lz, const double* __restrict__ w1,
                            const double* __restrict__ w2, const int* __restrict__ l0, double* __restrict__ ab,
                            unsigned char* __restrict__ piv)
{
    const int nxh = nx / 2 + 1;
    const long long Nk = (long long)nz * nxh;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nk) return;
    const int kz_i = (int)(k / nxh), kx_i = (int)(k - (long long)kz_i * nxh);
    const double k2 = ktrue2(kx_i, nx, Lx) + ktrue2(kz_i, nz, Lz);
    for (int r = 0; r < ny; ++r)
        for (int c = 0; c < S1_W; ++c) ab[((long long)r * S1_W + c) * Nk + k] = 0.0;
    for (int r = 0; r < ny; ++r) {
        const bool wall = (r == 0 || r == ny - 1);
        for (int l = 0; l < 5; ++l) band(ab, Nk, k, r, l0[r] + l) = wall ? w1[5 * r + l] : w2[5 * r + l];
        if (!wall) band(ab, Nk, k, r, r) -= k2;
    }
    if (k2 == 0.0) {                                  // p(y_0) = 0
        for (int l = 0; l < 5; ++l) band(ab, Nk, k, 0, l) = 0.0;
        band(ab, Nk, k, 0, 0) = 1.0;
    }
    for (int j = 0; j < ny; ++j) {
        const int rmax = min(j + S1_KL, ny - 1), cmax = min(j + S1_KL + S1_KU, ny - 1);
        int p = j;
        double best = fabs(band(ab, Nk, k, j, j));
        for (int r = j + 1; r <= rmax; ++r) {
            const double a = fabs(band(ab, Nk, k, r, j));
            if (a > best) { best = a; p = r; }
        }
        piv[(long long)j * Nk + k] = (unsigned char)(p - j);
        if (p != j)
            for (int c = j; c <= cmax; ++c) {
                const double t = band(ab, Nk, k, j, c);
                band(ab, Nk, k, j, c) = band(ab, Nk, k, p, c);
                band(ab, Nk, k, p, c) = t;
            }
        const double d = band(ab, Nk, k, j, j);
        for (int r = j + 1; r <= rmax; ++r) {
            const double m = band(ab, Nk, k, r, j) / d;
            band(ab, Nk, k, r, j) = m;
            if (m != 0.0)
                for (int c = j + 1; c <= cmax; ++c) band(ab, Nk, k, r, c) -= m * band(ab, Nk, k, j, c);
        }
    }
}

// Source, wall values and the banded solve of one snapshot: P[6][ny][Nk]
// (product spectra uu, uv, uw, vv, vw, ww), v = the snapshot's v spectra;
// writes p into pout[ny][Nk]
__global__ void k_s1_poisson(const zd* __restrict__ P, const zd* __restrict__ v, int ny, int nz, int nx, double Lx,
                             double Lz, double nu, const double* __restrict__ w1, const double* __restrict__ w2,
                             const int* __restrict__ l0, const double* __restrict__ ab,
                             const unsigned char* __restrict__ piv, zd* __restrict__ pout)
{
    const int nxh = nx / 2 + 1;
    const long long Nk = (long long)nz * nxh, fs = (long long)ny * Nk;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nk) return;
    const int kz_i = (int)(k / nxh), kx_i = (int)(k - (long long)kz_i * nxh);
    const double kx = kodd(kx_i, nx, Lx), kz = kodd(kz_i, nz, Lz);
    const double kx2 = ktrue2(kx_i, nx, Lx), kz2 = ktrue2(kz_i, nz, Lz), k2 = kx2 + kz2;
    auto at = [&](const zd* a, int r) { return a[(long long)r * Nk + k]; };
    auto stencil = [&](const double* w, const zd* a, int r) {
        zd s = mk(0.0, 0.0);
        for (int l = 0; l < 5; ++l) {
            const zd b = at(a, l0[r] + l);
            s = mk(s.x + w[5 * r + l] * b.x, s.y + w[5 * r + l] * b.y);
        }
        return s;
    };
    const zd *Puu = P, *Puv = P + fs, *Puw = P + 2 * fs, *Pvv = P + 3 * fs, *Pvw = P + 4 * fs, *Pww = P + 5 * fs;
    for (int r = 0; r < ny; ++r) {
        zd b;
        if (r == 0 || r == ny - 1) {
            const zd d2v = stencil(w2, v, r);
            b = (r == 0 && k2 == 0.0) ? mk(0.0, 0.0) : mk(nu * d2v.x, nu * d2v.y);
        } else {
            // d_i d_j (u_i u_j) = -kx^2 uu - kz^2 ww + (vv)'' - 2 kx kz uw + 2 i kx (uv)' + 2 i kz (vw)'
            const zd uu = at(Puu, r), ww = at(Pww, r), uw = at(Puw, r);
            const zd vv2 = stencil(w2, Pvv, r), uv1 = stencil(w1, Puv, r), vw1 = stencil(w1, Pvw, r);
            const double dx = -kx2 * uu.x - kz2 * ww.x + vv2.x - 2.0 * kx * kz * uw.x - 2.0 * (kx * uv1.y + kz * vw1.y);
            const double dy = -kx2 * uu.y - kz2 * ww.y + vv2.y - 2.0 * kx * kz * uw.y + 2.0 * (kx * uv1.x + kz * vw1.x);
            b = mk(-dx, -dy);
        }
        pout[(long long)r * Nk + k] = b;
    }
    // forward substitution with the row exchanges, then back substitution
    for (int j = 0; j < ny; ++j) {
        const int p = j + piv[(long long)j * Nk + k];
        zd bj = pout[(long long)p * Nk + k];
        if (p != j) {
            pout[(long long)p * Nk + k] = pout[(long long)j * Nk + k];
            pout[(long long)j * Nk + k] = bj;
        }
        const int rmax = min(j + S1_KL, ny - 1);
        for (int r = j + 1; r <= rmax; ++r) {
            const double m = ab[((long long)r * S1_W + (j - r + S1_KL)) * Nk + k];
            if (m != 0.0) {
                zd br = pout[(long long)r * Nk + k];
                pout[(long long)r * Nk + k] = mk(br.x - m * bj.x, br.y - m * bj.y);
            }
        }
    }
    for (int j = ny - 1; j >= 0; --j) {
        zd s = pout[(long long)j * Nk + k];
        const int cmax = min(j + S1_KL + S1_KU, ny - 1);
        for (int c = j + 1; c <= cmax; ++c) {
            const double a = ab[((long long)j * S1_W + (c - j + S1_KL)) * Nk + k];
            const zd x = pout[(long long)c * Nk + k];
            s = mk(s.x - a * x.x, s.y - a * x.y);
        }
        const double d = ab[((long long)j * S1_W + S1_KL) * Nk + k];
        pout[(long long)j * Nk + k] = mk(s.x / d, s.y / d);
    }
}

// ------------------------------------------------------------ launchers
size_t s1_band_doubles(int ny, long long Nk) { return (size_t)ny * S1_W * (size_t)Nk; }

static int col_nc(int nz) { return nz <= 256 ? 8 : 4; }
static size_t col_smem(int nz) { return (size_t)(1 + 2 * col_nc(nz)) * nz * sizeof(zd); }
static size_t row_smem(int nx) { return (size_t)7 * nx * sizeof(zd); }

cudaError_t s1_set_attrs(int nx, int nz)
{
    cudaError_t e = cudaFuncSetAttribute((const void*)k_s1_col<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)col_smem(nz));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)k_s1_col<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)col_smem(nz));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)k_s1_row_products, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)row_smem(nx));
    return e;
}

int s1_factor_launch(int ny, int nz, int nx, double Lx, double Lz, const double* w1, const double* w2, const int* l0,
                     double* ab, unsigned char* piv, cudaStream_t st)
{
    const long long Nk = (long long)nz * (nx / 2 + 1);
    k_s1_factor<<<(unsigned)((Nk + 127) / 128), 128, 0, st>>>(ny, nz, nx, Lx, Lz, w1, w2, l0, ab, piv);
    return 1;
}

int s1_snapshot_launch(const zd* v_eta, const double* mean_uw, int ny, int nz, int nx, double Lx, double Lz,
                       double nu, const double* w1, const double* w2, const int* l0, const zd* tw_x, const zd* tw_z,
                       const double* ab, const unsigned char* piv, zd* bufA, zd* bufB, zd* out, cudaStream_t st)
{
    const int nxh = nx / 2 + 1;
    const long long Nk = (long long)nz * nxh, fs = (long long)ny * Nk;
    const long long n = (long long)ny * Nk;
    k_s1_velocity<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v_eta, v_eta + fs, mean_uw, ny, nz, nx, Lx, Lz, w1,
                                                               l0, out);
    const int nc = col_nc(nz);
    dim3 gc((unsigned)((nxh + nc - 1) / nc), (unsigned)ny, 3);
    k_s1_col<true><<<gc, 256, col_smem(nz), st>>>(out, ny, nz, nxh, nc, tw_z, bufA);
    k_s1_row_products<<<dim3((unsigned)nz, (unsigned)ny), 256, row_smem(nx), st>>>(bufA, ny, nz, nx, tw_x, bufB);
    gc.z = 6;
    k_s1_col<false><<<gc, 256, col_smem(nz), st>>>(bufB, ny, nz, nxh, nc, tw_z, bufA);
    k_s1_poisson<<<(unsigned)((Nk + 127) / 128), 128, 0, st>>>(bufA, out + fs, ny, nz, nx, Lx, Lz, nu, w1, w2, l0, ab,
                                                               piv, out + 3 * fs);
    return 5;
}

}  // namespace gke
