// gke_combine.cu -- per-pair term spectra from one batch's contractions.
//
// Every GKE term is one inverse transform of a linear combination of the
// contraction spectra plus a part that depends on (Y1, Y2) only (correlation
// expansion, Sec. 3.1 Eq. 7; Parseval, Eq. 8-9).  With X^H(y, y') =
// conj X(y', y), S0 = D, S1 = E + E^H, S2 = E^H - E, S3 = F + F^H,
// S4 = Gx - Gx^H, S5 = Gy - Gy^H, S6 = Gz - Gz^H, S7 = H + H^H, where
// Gy = QV + X2 and H = QV - X2:
//   A     : -2 S0
//   Phi_x : S4 + (-2 dU + 4 i nu kx) S0
//   Phi_y : S5
//   Phi_z : S6 + 4 i nu kz S0
//   phi   : S7 / 2 - 2 S3
//   xi    : 2 U'* S1 - dU' S2
//   res   : i kx S4 + i kz S6 - 2 i dU kx S0 - 4 nu |k|^2 S0 - xi
// (dU = U(Y2) - U(Y1), U'* = (U'(Y1) + U'(Y2))/2, dU' = U'(Y2) - U'(Y1), kx,
// kz the signed wavenumbers with 0 on the Nyquist lines).  The combinations
// are linear in the contractions and their coefficients depend only on the
// mean (frozen before the first batch), so batches are summed here:
//   comb[p][t][k] (+)= T_t(p, k)
// with the arithmetic in TC and the sum in TO: double / double on the plain
// path; on the split path float / float for the first batch and float /
// double once a second batch arrives (the per-pair sum is then promoted to
// FP64 by k_promote).
//
// CTA = an 8 x 8 block of pairs (i1 in [8a, 8a+8), i2 in [8b, 8b+8), b >= a)
// and KC consecutive wavenumbers.  In the raw layout the block (a, b) of a
// contraction over KC wavenumbers is KC x 64 contiguous values, and so is the
// transposed partner block (b, a); both are staged through shared memory, then
// each thread forms the terms of its (pair, k) items; stores are k-contiguous.
#include <algorithm>

#include "gke_common.cuh"
#include "gke_kernels.h"

namespace gke {

constexpr int PB = 8;     // pair block edge
constexpr int CHUNKS = 1; // k chunks per CTA

// KC = wavenumbers per CTA.  Default: ~30 KB of staging per CTA, so several
// CTAs per SM hide the gather latency; the plan's tuner may pick another of
// the instantiated widths (combine_kc_ok).
template <typename TI> struct CombCfg;
template <> struct CombCfg<float> { static constexpr int KC = 4; };
template <> struct CombCfg<double> { static constexpr int KC = 2; };

// Staging layout, in complex values: block (slot, q) every SQ, row rr every
// SR, column cc contiguous.  With SR odd and SQ = 4 mod 16 the item reads of
// a half-warp (4 wavenumbers q x 4 columns m of a row, or the transposed
// partner: 4 q x 4 rows m) hit 16 distinct 8-byte bank pairs (FP32 values),
// and the 8 reads of a quarter-warp distinct 16-byte ones (FP64, 2 q x 4 m).
constexpr int SR = PB + 1, SQ = 84;
static_assert(SQ >= PB * SR && SQ % 16 == 4 && SR % 2 == 1, "combine staging layout");

template <typename TI, int KC> constexpr size_t combine_smem_bytes()
{
    return (size_t)(2 * NJOB - 1) * KC * SQ * sizeof(cplx<TI>);
}
int combine_kc(bool fp32) { return fp32 ? CombCfg<float>::KC : CombCfg<double>::KC; }
bool combine_kc_ok(bool fp32, int kc) { return fp32 ? (kc == 2 || kc == 4 || kc == 8) : (kc == 1 || kc == 2 || kc == 4); }

// The seven term spectra of one (pair, wavenumber) from the contractions
// x12[j] = X_j(Y1, Y2) and x21[j] = conj X_j(Y2, Y1) (D has no partner).
template <typename TC>
__device__ __forceinline__ void pair_terms(const cplx<TC>* x12, const cplx<TC>* x21, TC kx, TC kz, TC dU, TC Upm,
                                           TC dUp, TC nuc, cplx<TC>* T)
{
    typedef cplx<TC> Z;
    const Z S0 = x12[J_D];
    const Z S1 = x12[J_E] + x21[J_E], S2 = x21[J_E] - x12[J_E];
    const Z S3 = x12[J_F] + x21[J_F];
    const Z S4 = x12[J_GX] - x21[J_GX];
    const Z S6 = x12[J_GZ] - x21[J_GZ];
    const Z S5 = (x12[J_QV] + x12[J_X]) - (x21[J_QV] + x21[J_X]);
    const Z S7 = (x12[J_QV] - x12[J_X]) + (x21[J_QV] - x21[J_X]);
    T[T_A] = (TC)(-2) * S0;
    T[T_PHIX] = S4 + ((TC)(-2) * dU) * S0 + ((TC)4 * nuc * kx) * mul_i(S0);
    T[T_PHIY] = S5;
    T[T_PHIZ] = S6 + ((TC)4 * nuc * kz) * mul_i(S0);
    T[T_PHI] = (TC)0.5 * S7 - (TC)2 * S3;
    T[T_XI] = ((TC)2 * Upm) * S1 - dUp * S2;
    T[T_RES] = kx * mul_i(S4) + kz * mul_i(S6) + ((TC)(-2) * dU * kx) * mul_i(S0)
             + ((TC)(-4) * nuc * (kx * kx + kz * kz)) * S0 - T[T_XI];
}

template <typename TI, typename TC, typename TO, int KC>
__global__ void __launch_bounds__(256)
k_combine(const cplx<TI>* __restrict__ raw, int ny, int nz, int nx, double Lx, double Lz, double nu,
          const double* __restrict__ prof, int beta, int kbase, int Kc, long long cstride, unsigned tmask,
          unsigned jmask, cplx<TO>* __restrict__ comb)
{
    typedef cplx<TI> C;
    typedef cplx<TC> Z;
    extern __shared__ __align__(16) unsigned char sh_raw_cb[];
    // stage[slot][q][rr][cc]: slot 2 j = block of job j, 2 j + 1 = partner block
    // (rows y in [8b, 8b+8), columns y' in [8a, 8a+8)); D has no partner slot
    C* stage = (C*)sh_raw_cb;
    // this launch covers the wavenumbers [kbase, kbase + Kc): raw holds them
    // (chunk-local index kl), comb rows are cstride long from kl = 0
    const int nxh = nx / 2 + 1, Nk = Kc;
    const int nblk = (ny + PB - 1) / PB;
    int bt = blockIdx.y, a = 0;
    while (bt >= nblk - a) { bt -= nblk - a; ++a; }
    const int b = a + bt;
    const int nslot = 2 * NJOB - 1;
    auto at = [&](int slot, int q, int rr, int cc) -> C& {
        return stage[(slot * KC + q) * SQ + rr * SR + cc];
    };
    // per-wavenumber and per-pair coefficients, formed once per CTA (FP64
    // arithmetic costs as much as ~60 FP32 operations here, so none is done
    // per item)
    __shared__ TC s_kx[KC], s_kz[KC];
    __shared__ TC s_dU[PB * PB], s_Upm[PB * PB], s_dUp[PB * PB];
    if (threadIdx.x < PB * PB) {
        const int i1 = min(PB * a + threadIdx.x / PB, ny - 1), i2 = min(PB * b + threadIdx.x % PB, ny - 1);
        s_dU[threadIdx.x] = (TC)(prof[PR_U * ny + i2] - prof[PR_U * ny + i1]);
        s_Upm[threadIdx.x] = (TC)(0.5 * (prof[PR_DU * ny + i1] + prof[PR_DU * ny + i2]));
        s_dUp[threadIdx.x] = (TC)(prof[PR_DU * ny + i2] - prof[PR_DU * ny + i1]);
    }
    // each CTA walks CHUNKS consecutive chunks of KC wavenumbers
    for (int ch = 0; ch < CHUNKS; ++ch) {
    const int k0 = (blockIdx.x * CHUNKS + ch) * KC;
    if (k0 >= Nk) break;
    __syncthreads();
    if (threadIdx.x >= 256 - KC) {
        const int kk = threadIdx.x - (256 - KC), k = kbase + min(k0 + kk, Nk - 1);
        const int kz_i = k / nxh, kx_i = k - kz_i * nxh;
        s_kx[kk] = (TC)(6.283185307179586476925286766559 * signed_bin(kx_i, nx) / Lx);
        s_kz[kk] = (TC)(6.283185307179586476925286766559 * signed_bin(kz_i, nz) / Lz);
    }
    // two consecutive values per thread (one 16-byte load on the split path)
    for (int e = threadIdx.x; e < nslot * KC * PB * PB / 2; e += blockDim.x) {
        const int e2 = 2 * e;
        const int slot = e2 / (KC * PB * PB);
        const int rem = e2 - slot * KC * PB * PB;
        const int q = rem / (PB * PB), rr = (rem / PB) % PB, cc = rem % PB;
        const int j = slot >> 1, partner = slot & 1;
        const int kq = k0 + q;
        const int yb = partner ? b : a, ypb = partner ? a : b;
        C v0 = mk((TI)0, (TI)0), v1 = v0;
        if (kq < Nk && ((jmask >> j) & 1u)) {         // contractions outside the term set stay zero
            const C* src = raw + ((((long long)j * nblk + yb) * nblk + ypb) * Nk + kq) * 64 + rr * PB + cc;
            if (sizeof(C) == 8) {
                const float4 f4 = __ldcs((const float4*)src);
                v0 = *(const C*)&f4.x;
                v1 = *(const C*)&f4.z;
            } else {
                v0 = src[0];
                v1 = src[1];
            }
        }
        at(slot, q, rr, cc) = v0;
        at(slot, q, rr, cc + 1) = v1;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < KC * PB * PB; it += blockDim.x) {
        const int kk = it % KC, pm = it / KC, r = pm / PB, m = pm % PB;
        const int k = k0 + kk, i1 = PB * a + r, i2 = PB * b + m;
        if (k >= Nk || i1 >= ny || i2 >= ny || i2 < i1) continue;
        const TC kx = s_kx[kk], kz = s_kz[kk];
        const TC dU = s_dU[pm], Upm = s_Upm[pm], dUp = s_dUp[pm];
        Z x12[NJOB], x21[NJOB];
        #pragma unroll
        for (int j = 0; j < NJOB; ++j) {
            const C v = at(2 * j, kk, r, m);
            x12[j] = mk((TC)v.x, (TC)v.y);
            if (j != J_D) {
                const C w = at(2 * j + 1, kk, m, r);
                x21[j] = mk((TC)w.x, -(TC)w.y);                           // conj
            } else {
                x21[j] = mk((TC)0, (TC)0);
            }
        }
        Z T[NTERM];
        pair_terms<TC>(x12, x21, kx, kz, dU, Upm, dUp, (TC)nu, T);
        cplx<TO>* dst = comb + pair_index(i1, i2, ny) * NTERM * cstride + k;
        #pragma unroll
        for (int t = 0; t < NTERM; ++t) {
            if (!((tmask >> t) & 1u)) continue;
            cplx<TO> v = mk((TO)T[t].x, (TO)T[t].y);
            if (beta) {
                v = v + dst[(long long)t * cstride];
                dst[(long long)t * cstride] = v;
            } else {
                st_stream(dst + (long long)t * cstride, v);
            }
        }
    }
    }
}

// comb64[i] = comb32[i] (promotion of the first batch's per-pair sums)
__global__ void k_promote(const zf* __restrict__ src, long long n, zd* __restrict__ dst)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = mk((double)src[i].x, (double)src[i].y);
}

// Mirror sampling (Sec. 3.2 Step 2, Sec. 3.3): the spectra of the wedge pair
// (i1, i2) averaged with those of the snapshots' mirror images.  A mirror
// image's term at (i1, i2, r) equals sigma_t times the snapshot's term at
// (ny-1-i2, ny-1-i1, -r) (combined inversion of y and r), and r -> -r
// conjugates the spectrum of a real field, so
//   out[pw][t][k] = (comb[p][t][k] + sigma_t conj(comb[p'][t][k])) / 2,
// p = (i1, i2), p' = (ny-1-i2, ny-1-i1) in the triangle's pair order.
__constant__ float c_sigma[NTERM] = {1.f, -1.f, 1.f, -1.f, -1.f, 1.f, 1.f};

template <typename T>
__global__ void k_mirror_fold(const cplx<T>* __restrict__ comb, const int* __restrict__ pair_w, int ny, int Nk,
                              cplx<T>* __restrict__ out)
{
    const long long row = blockIdx.x;                 // pw * NTERM + t
    const long long pw = row / NTERM;
    const int t = (int)(row - pw * NTERM);
    const int i1 = pair_w[2 * pw], i2 = pair_w[2 * pw + 1];
    const cplx<T>* a = comb + (pair_index(i1, i2, ny) * NTERM + t) * (long long)Nk;
    const cplx<T>* b = comb + (pair_index(ny - 1 - i2, ny - 1 - i1, ny) * NTERM + t) * (long long)Nk;
    cplx<T>* o = out + row * (long long)Nk;
    const T sg = (T)c_sigma[t], h = (T)0.5;
    for (int k = blockIdx.y * blockDim.x + threadIdx.x; k < Nk; k += gridDim.y * blockDim.x) {
        const cplx<T> va = ld_stream(a + k), vb = ld_stream(b + k);
        st_stream(o + k, mk(h * (va.x + sg * vb.x), h * (va.y - sg * vb.y)));
    }
}

int mirror_fold_launch(bool c64, const void* comb, const int* pair_w, long long nout, int ny, int Nk, void* out,
                       cudaStream_t st)
{
    dim3 g((unsigned)(nout * NTERM), (unsigned)std::min(8, (Nk + 255) / 256));
    if (c64)
        k_mirror_fold<double><<<g, 256, 0, st>>>((const zd*)comb, pair_w, ny, Nk, (zd*)out);
    else
        k_mirror_fold<float><<<g, 256, 0, st>>>((const zf*)comb, pair_w, ny, Nk, (zf*)out);
    return 1;
}

// Uniform undersampling of the separations by s_z x s_x (Sec. 3.4), exact by
// aliasing: the term at r = (s_z m_z, s_x m_x) is the inverse transform, on
// the coarse nzd x nxd grid (nzd = nz / s_z, nxd = nx / s_x), of the spectrum
//   G(kzd, kxd) = sum of F_H(kz, kx) over kz = kzd (mod nzd), kx = kxd (mod nxd),
// F_H the Hermitian extension of the stored half spectrum (its kx = 0 and
// kx = nx/2 columns taken as their Hermitian parts, as the full-size inverse
// transform does).  So a stored value F(kz, kx), 0 <= kx <= nx/2, adds
// h F to the bin (kz, kx) and h conj F to the bin (-kz, -kx) (mod nzd, nxd),
// h = 1/2 on the columns kx = 0 and nx/2, else 1.
//
// The contractions run in chunks of whole conjugate classes of kz rows,
// {kz : kz mod nzd in {c, -c}}: every source of the coarse rows c and -c then
// lies in one chunk, and the FP64 coarse spectra of a row are read and
// written once per batch.

// dst[f][kl][e] = src[f][rows[i] nxh + kx][e], kl = i nxh + kx: the chunk's
// wavenumbers gathered into a contiguous operand set (per_k values each)
template <typename T>
__global__ void k_gather_rows(const T* __restrict__ src, long long Nk, long long per_k, const int* __restrict__ rows,
                              int nrows, int nxh, T* __restrict__ dst)
{
    const int i = blockIdx.x, f = blockIdx.y;
    const long long n = (long long)nxh * per_k;
    const T* s = src + ((long long)f * Nk + (long long)rows[i] * nxh) * per_k;
    T* d = dst + ((long long)f * nrows * nxh + (long long)i * nxh) * per_k;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) d[e] = s[e];
}

int gather_rows_launch(bool c64, const void* src, int nf, long long Nk, long long per_k, const int* rows, int nrows,
                       int nxh, void* dst, cudaStream_t st)
{
    dim3 g((unsigned)nrows, (unsigned)nf);
    if (c64) k_gather_rows<zd><<<g, 256, 0, st>>>((const zd*)src, Nk, per_k, rows, nrows, nxh, (zd*)dst);
    else k_gather_rows<zf><<<g, 256, 0, st>>>((const zf*)src, Nk, per_k, rows, nrows, nxh, (zf*)dst);
    return 1;
}

// FP32 sums are compensated (Kahan), FP64 ones plain
template <typename TC> struct Acc {
    cplx<TC> s;
    __device__ __forceinline__ void zero() { s = mk((TC)0, (TC)0); }
    __device__ __forceinline__ void add(cplx<TC> v) { s = s + v; }
    __device__ __forceinline__ double re() const { return (double)s.x; }
    __device__ __forceinline__ double im() const { return (double)s.y; }
};
template <> struct Acc<float> {
    float sx, sy, cx, cy;
    __device__ __forceinline__ void zero() { sx = sy = cx = cy = 0.f; }
    __device__ __forceinline__ static void kahan(float& s, float& c, float v)
    {
        const float y = __fsub_rn(v, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ void add(zf v) { kahan(sx, cx, v.x); kahan(sy, cy, v.y); }
    __device__ __forceinline__ double re() const { return (double)sx - (double)cx; }
    __device__ __forceinline__ double im() const { return (double)sy - (double)cy; }
};

// One chunk's contractions -> the term spectra of every triangle pair ->
// their coarse bins, added to dec[p][t][kzd][kxd] (FP64).  CTA = the 64
// pairs of an 8 x 8 block (a, b), b >= a, times FK coarse columns kxd;
// a thread owns one (pair, kxd) and walks the chunk's coarse rows, summing
// for each the direct sources (kz = kzd, kx = kxd) and the conjugate images
// (kz = -kzd, kx = -kxd) of the chunk's rows.  The 32 lanes of a warp are
// 32 pairs of the block, so every contraction load is one contiguous
// 256-byte row of the raw layout (the partner block's: 8 sectors).
constexpr int FK = 4;
template <typename TI, typename TC>
__global__ void __launch_bounds__(64 * FK)
k_combine_fold(const cplx<TI>* __restrict__ raw, const int* __restrict__ rows, int nrows,
               const int* __restrict__ crs, int ncr, int ny, int nz, int nx, int nzd, int nxd, double Lx, double Lz,
               double nu, const double* __restrict__ prof, unsigned tmask, unsigned jmask, zd* __restrict__ dec)
{
    typedef cplx<TI> C;
    typedef cplx<TC> Z;
    extern __shared__ int sh_cf[];                    // per chunk row: direct and image coarse rows
    const int nxh = nx / 2 + 1, nxdh = nxd / 2 + 1, Kc = nrows * nxh;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        sh_cf[i] = rows[i] % nzd;
        sh_cf[nrows + i] = (nz - rows[i]) % nzd;
    }
    __syncthreads();
    const int nblk = (ny + PB - 1) / PB;
    int bt = blockIdx.x, a = 0;
    while (bt >= nblk - a) { bt -= nblk - a; ++a; }
    const int b = a + bt;
    const int pm = threadIdx.x & 63, r = pm >> 3, m = pm & 7;
    const int kxd = blockIdx.y * FK + (threadIdx.x >> 6);
    const int i1 = PB * a + r, i2 = PB * b + m;
    if (kxd >= nxdh || i1 >= ny || i2 >= ny || i2 < i1) return;
    const TC dU = (TC)(prof[PR_U * ny + i2] - prof[PR_U * ny + i1]);
    const TC Upm = (TC)(0.5 * (prof[PR_DU * ny + i1] + prof[PR_DU * ny + i2]));
    const TC dUp = (TC)(prof[PR_DU * ny + i2] - prof[PR_DU * ny + i1]);
    const TC cx = (TC)(6.283185307179586476925286766559 / Lx), cz = (TC)(6.283185307179586476925286766559 / Lz);
    const TC nuc = (TC)nu;
    const long long jstride = (long long)nblk * nblk * Kc * 64;
    const C* p12 = raw + ((long long)a * nblk + b) * Kc * 64 + pm;          // block (a, b), element (r, m)
    const C* p21 = raw + ((long long)b * nblk + a) * Kc * 64 + m * PB + r;  // block (b, a), element (m, r)
    const int kxm = (nxd - kxd) % nxd;                   // -kxd mod nxd
    zd* out = dec + pair_index(i1, i2, ny) * NTERM * (long long)nzd * nxdh + kxd;
    for (int ci = 0; ci < ncr; ++ci) {
        const int kzd = crs[ci];
        Acc<TC> acc[NTERM];
        #pragma unroll
        for (int t = 0; t < NTERM; ++t) acc[t].zero();
        for (int i = 0; i < nrows; ++i) {
            const bool direct = sh_cf[i] == kzd, image = sh_cf[nrows + i] == kzd;
            if (!direct && !image) continue;
            const int kz = rows[i];
            const TC kzv = cz * (TC)signed_bin(kz, nz);
            // direct sources kx = kxd (mod nxd), then the images kx = -kxd
            for (int pass = 0; pass < 2; ++pass) {
                if (!(pass ? image : direct)) continue;
                for (int kx = pass ? kxm : kxd; 2 * kx <= nx; kx += nxd) {
                    const long long kl = (long long)i * nxh + kx;
                    Z x12[NJOB], x21[NJOB];
                    #pragma unroll
                    for (int j = 0; j < NJOB; ++j) {
                        C v = mk((TI)0, (TI)0), w = v;
                        if ((jmask >> j) & 1u) {
                            v = p12[j * jstride + kl * 64];
                            if (j != J_D) w = p21[j * jstride + kl * 64];
                        }
                        x12[j] = mk((TC)v.x, (TC)v.y);
                        x21[j] = mk((TC)w.x, -(TC)w.y);
                    }
                    Z T[NTERM];
                    pair_terms<TC>(x12, x21, cx * (TC)signed_bin(kx, nx), kzv, dU, Upm, dUp, nuc, T);
                    const TC h = (kx == 0 || 2 * kx == nx) ? (TC)0.5 : (TC)1;
                    #pragma unroll
                    for (int t = 0; t < NTERM; ++t)
                        acc[t].add(mk(h * T[t].x, pass ? -h * T[t].y : h * T[t].y));
                }
            }
        }
        #pragma unroll
        for (int t = 0; t < NTERM; ++t) {
            if (!((tmask >> t) & 1u)) continue;
            zd* o = out + ((long long)t * nzd + kzd) * nxdh;
            zd v = *o;
            v.x += acc[t].re();
            v.y += acc[t].im();
            *o = v;
        }
    }
}

int combine_fold_launch(bool c64, const void* raw, const int* rows, int nrows, const int* crs, int ncr, int ny,
                        int nz, int nx, int nzd, int nxd, double Lx, double Lz, double nu, const double* prof,
                        unsigned tmask, void* dec, cudaStream_t st)
{
    const int nblk = (ny + PB - 1) / PB, nxdh = nxd / 2 + 1;
    dim3 g((unsigned)(nblk * (nblk + 1) / 2), (unsigned)((nxdh + FK - 1) / FK));
    const unsigned jm = job_set(tmask);
    if (c64)
        k_combine_fold<double, double><<<g, 64 * FK, (size_t)2 * nrows * sizeof(int), st>>>((const zd*)raw, rows, nrows, crs, ncr, ny, nz, nx, nzd,
                                                              nxd, Lx, Lz, nu, prof, tmask, jm, (zd*)dec);
    else
        k_combine_fold<float, float><<<g, 64 * FK, (size_t)2 * nrows * sizeof(int), st>>>((const zf*)raw, rows, nrows, crs, ncr, ny, nz, nx, nzd,
                                                            nxd, Lx, Lz, nu, prof, tmask, jm, (zd*)dec);
    return 1;
}

// Chunked mode on the split path in plane mode: the chunk's six plane
// spectra planes[NPLANE][Kc][npp] (FP32, pair index fastest) give the seven
// term spectra of a triangle pair as the transforms' column pass forms them
// (Phi_x = S4 + (dU - 2 i nu kx) A, Phi_z = S6 - 2 i nu kz A, residual =
// i kx Phi_x + i kz Phi_z - xi), which are aliased onto the coarse grid as in
// k_combine_fold.  CTA = 128 consecutive pairs x 2 adjacent coarse columns:
// four warps read 1 KB of one plane row at a time and the two columns' FP64
// coarse bins fill whole 32-byte sectors.  The chunk rows that feed each
// coarse row (direct and image) are listed once per CTA in shared memory.
constexpr int PF_PAIRS = 128, PF_COLS = 2;
__global__ void __launch_bounds__(PF_PAIRS * PF_COLS)
k_planes_fold(const zf* __restrict__ planes, long long npp, int Kc, const int* __restrict__ rows, int nrows,
              const int* __restrict__ crs, int ncr, const int* __restrict__ pair_tri, long long npair, int ny, int nz,
              int nx, int nzd, int nxd, double Lx, double Lz, double nu, const double* __restrict__ prof,
              unsigned tmask, zd* __restrict__ dec)
{
    // src[ci][j]: chunk row i * 2 + pass (0 direct, 1 image) of coarse row ci,
    // cnt[ci] <= 2 nz / nzd of them (a coarse row has nz / nzd direct rows and
    // as many images, all in its chunk)
    extern __shared__ int sh_pf[];
    const int ms = 2 * (nz / nzd);
    int* cnt = sh_pf;
    int* src = sh_pf + ncr;
    const int nxh = nx / 2 + 1, nxdh = nxd / 2 + 1;
    for (int ci = threadIdx.x; ci < ncr; ci += blockDim.x) {
        const int kzd = crs[ci];
        int n = 0;
        for (int i = 0; i < nrows && n < ms; ++i) {
            if (rows[i] % nzd == kzd) src[ci * ms + n++] = i * 2;
            if ((nz - rows[i]) % nzd == kzd && n < ms) src[ci * ms + n++] = i * 2 + 1;
        }
        cnt[ci] = n;
    }
    __syncthreads();
    const long long p = (long long)blockIdx.x * PF_PAIRS + (threadIdx.x % PF_PAIRS);
    const int kxd = blockIdx.y * PF_COLS + (int)(threadIdx.x / PF_PAIRS);
    if (p >= npair || kxd >= nxdh) return;
    const int i1 = pair_tri[2 * p], i2 = pair_tri[2 * p + 1];
    const float dU = (float)(prof[PR_U * ny + i2] - prof[PR_U * ny + i1]);
    const float cx = (float)(6.283185307179586476925286766559 / Lx), cz = (float)(6.283185307179586476925286766559 / Lz);
    const float nu2 = (float)(2.0 * nu);
    const int kxm = (nxd - kxd) % nxd;                   // -kxd mod nxd
    const long long pstride = (long long)Kc * npp;
    zd* out = dec + p * NTERM * (long long)nzd * nxdh + kxd;
    for (int ci = 0; ci < ncr; ++ci) {
        const int kzd = crs[ci];
        Acc<float> acc[NTERM];
        #pragma unroll
        for (int t = 0; t < NTERM; ++t) acc[t].zero();
        for (int j = 0; j < cnt[ci]; ++j) {
            const int e = src[ci * ms + j], i = e >> 1, pass = e & 1;
            const float kzv = cz * (float)signed_bin(rows[i], nz);
            // direct sources kx = kxd (mod nxd), images kx = -kxd
            for (int kx = pass ? kxm : kxd; 2 * kx <= nx; kx += nxd) {
                const zf* q = planes + ((long long)i * nxh + kx) * npp + p;
                const zf A = q[PL_A * pstride], S4 = q[PL_S4 * pstride], PY = q[PL_PHIY * pstride];
                const zf S6 = q[PL_S6 * pstride], PH = q[PL_PHI * pstride], XI = q[PL_XI * pstride];
                const float kxv = cx * (float)signed_bin(kx, nx);
                const zf PX = mk(S4.x + dU * A.x + nu2 * kxv * A.y, S4.y + dU * A.y - nu2 * kxv * A.x);
                const zf PZ = mk(S6.x + nu2 * kzv * A.y, S6.y - nu2 * kzv * A.x);
                const zf RS = mk(-kxv * PX.y - kzv * PZ.y - XI.x, kxv * PX.x + kzv * PZ.x - XI.y);
                const zf T[NTERM] = {A, PX, PY, PZ, PH, XI, RS};
                const float h = (kx == 0 || 2 * kx == nx) ? 0.5f : 1.f;
                #pragma unroll
                for (int t = 0; t < NTERM; ++t) acc[t].add(mk(h * T[t].x, pass ? -h * T[t].y : h * T[t].y));
            }
        }
        #pragma unroll
        for (int t = 0; t < NTERM; ++t) {
            if (!((tmask >> t) & 1u)) continue;
            zd* o = out + ((long long)t * nzd + kzd) * nxdh;
            zd v = *o;
            v.x += acc[t].re();
            v.y += acc[t].im();
            *o = v;
        }
    }
}

int planes_fold_launch(const void* planes, long long npp, int Kc, const int* rows, int nrows, const int* crs, int ncr,
                       const int* pair_tri, long long npair, int ny, int nz, int nx, int nzd, int nxd, double Lx,
                       double Lz, double nu, const double* prof, unsigned tmask, void* dec, cudaStream_t st)
{
    const int nxdh = nxd / 2 + 1;
    dim3 g((unsigned)((npair + PF_PAIRS - 1) / PF_PAIRS), (unsigned)((nxdh + PF_COLS - 1) / PF_COLS));
    k_planes_fold<<<g, PF_PAIRS * PF_COLS, (size_t)(ncr + ncr * 2 * (nz / nzd)) * sizeof(int), st>>>((const zf*)planes, npp, Kc, rows, nrows, crs, ncr, pair_tri, npair, ny, nz, nx,
                                      nzd, nxd, Lx, Lz, nu, prof, tmask, (zd*)dec);
    return 1;
}

template <typename TI, typename TO, int KC>
static void combine_kc_launch(const void* raw, int ny, int nz, int nx, double Lx, double Lz, double nu,
                              const double* prof, int beta, int kbase, int Kc, long long cstride, void* comb,
                              unsigned terms, unsigned jobs, cudaStream_t st)
{
    const int kc = KC * CHUNKS;
    const int nblk = (ny + PB - 1) / PB;
    dim3 grid((Kc + kc - 1) / kc, nblk * (nblk + 1) / 2);
    k_combine<TI, TI, TO, KC><<<grid, 256, combine_smem_bytes<TI, KC>(), st>>>(
        (const cplx<TI>*)raw, ny, nz, nx, Lx, Lz, nu, prof, beta, kbase, Kc, cstride, terms, jobs, (cplx<TO>*)comb);
}

template <typename TI, typename TO>
static void combine_t(int kc, const void* raw, int ny, int nz, int nx, double Lx, double Lz, double nu,
                      const double* prof, int beta, int kbase, int Kc, long long cstride, void* comb,
                      unsigned terms, unsigned jobs, cudaStream_t st)
{
#define GKE_COMB_ARGS raw, ny, nz, nx, Lx, Lz, nu, prof, beta, kbase, Kc, cstride, comb, terms, jobs, st
    if constexpr (sizeof(TI) == 4) {
        if (kc == 2) combine_kc_launch<TI, TO, 2>(GKE_COMB_ARGS);
        else if (kc == 8) combine_kc_launch<TI, TO, 8>(GKE_COMB_ARGS);
        else combine_kc_launch<TI, TO, 4>(GKE_COMB_ARGS);
    } else {
        if (kc == 1) combine_kc_launch<TI, TO, 1>(GKE_COMB_ARGS);
        else if (kc == 4) combine_kc_launch<TI, TO, 4>(GKE_COMB_ARGS);
        else combine_kc_launch<TI, TO, 2>(GKE_COMB_ARGS);
    }
#undef GKE_COMB_ARGS
}

// comb (+)= term spectra of one batch.  fp32_in: raw and arithmetic in FP32;
// out64: comb is FP64 (else FP32); kc: wavenumbers per CTA (0 = default)
// wavenumbers [kbase, kbase + Kc) (raw holds that chunk); comb rows of
// cstride values per (pair, term), chunk-local index kl at offset kl
int combine_launch(bool fp32_in, bool out64, const void* raw, int ny, int nz, int nx, double Lx, double Lz,
                   double nu, const double* prof, int beta, int kbase, int Kc, long long cstride, void* comb,
                   unsigned terms, int kc, cudaStream_t st)
{
    const unsigned jobs = job_set(terms);
    if (!combine_kc_ok(fp32_in, kc)) kc = combine_kc(fp32_in);
    if (!fp32_in)
        combine_t<double, double>(kc, raw, ny, nz, nx, Lx, Lz, nu, prof, beta, kbase, Kc, cstride, comb, terms, jobs,
                                  st);
    else if (out64)
        combine_t<float, double>(kc, raw, ny, nz, nx, Lx, Lz, nu, prof, beta, kbase, Kc, cstride, comb, terms, jobs,
                                 st);
    else
        combine_t<float, float>(kc, raw, ny, nz, nx, Lx, Lz, nu, prof, beta, kbase, Kc, cstride, comb, terms, jobs,
                                st);
    return 1;
}

// Plane mode (split correlator on one 128-row tile): the batches' FP32 plane
// spectra summed in FP64, dst[j] = (beta ? dst[j] : 0) + src[j] for the
// selected planes j (per_plane complex values each); beta = 0 promotes the
// first batch before the second one is written over it
__global__ void k_planes_accum(const zf* __restrict__ src, long long per_plane, unsigned planes, int beta,
                               zd* __restrict__ dst)
{
    const int j = blockIdx.y;
    if (!((planes >> j) & 1u)) return;
    const zf* s = src + (long long)j * per_plane;
    zd* d = dst + (long long)j * per_plane;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per_plane;
         i += (long long)gridDim.x * blockDim.x) {
        const zf v = ld_stream(s + i);
        zd o = mk((double)v.x, (double)v.y);
        if (beta) o = o + d[i];
        st_stream(d + i, o);
    }
}

int planes_accum_launch(const void* src, long long per_plane, unsigned planes, int beta, void* dst, cudaStream_t st)
{
    k_planes_accum<<<dim3(152 * 4, NPLANE), 256, 0, st>>>((const zf*)src, per_plane, planes, beta, (zd*)dst);
    return 1;
}

int promote_launch(const void* comb32, long long n, void* comb64, cudaStream_t st)
{
    k_promote<<<152 * 8, 256, 0, st>>>((const zf*)comb32, n, (zd*)comb64);
    return 1;
}

cudaError_t combine_set_attrs()
{
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* k, size_t bytes) {
        const cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (r != cudaSuccess) e = r;
    };
    set((const void*)k_combine<double, double, double, 1>, combine_smem_bytes<double, 1>());
    set((const void*)k_combine<double, double, double, 2>, combine_smem_bytes<double, 2>());
    set((const void*)k_combine<double, double, double, 4>, combine_smem_bytes<double, 4>());
    set((const void*)k_combine<float, float, float, 2>, combine_smem_bytes<float, 2>());
    set((const void*)k_combine<float, float, float, 4>, combine_smem_bytes<float, 4>());
    set((const void*)k_combine<float, float, float, 8>, combine_smem_bytes<float, 8>());
    set((const void*)k_combine<float, float, double, 2>, combine_smem_bytes<float, 2>());
    set((const void*)k_combine<float, float, double, 4>, combine_smem_bytes<float, 4>());
    set((const void*)k_combine<float, float, double, 8>, combine_smem_bytes<float, 8>());
    return e;
}

}  // namespace gke
