// gke_common.cuh -- device helpers shared by the GKE kernels.
//
// Layout conventions of the Parseval path (all device memory, C order):
//   fields   complex [nsnap][4][ny][nz][nxh]   input Fourier coefficients of
//            u, v, w, p, forward-normalised: a_hat(k) = (1/(nx nz)) sum_x a e^{-ik.x}
//   Xop      complex [NFIELD][Nk][ns][ny]      correlator operands, one block
//            of ns x ny values per (field, wavenumber); Nk = nz * nxh,
//            k = kz_index * nxh + kx_index
//   acc_sq   complex [NJSQ][ny][ny][Nk]        per-wavenumber spectral sums of
//            the cross contractions, ordered pairs (y, y')
//   acc_D    complex [npair][Nk]               Hermitian contraction, pairs y <= y'
//   terms    double  [NTERM][npair][nz][nx]    GKE terms in separation space,
//            separation index (m_z, m_x) in FFT order, r = (m_x Lx/nx, m_z Lz/nz)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gke {

// correlated fields (Sec. 3.1: the linear fields and the in-plane products)
enum Field { F_U = 0, F_V, F_W, F_P, F_UU, F_VV, F_WW, F_UV, F_UW, F_VW, F_Q, NFIELD };
// cross contractions over snapshots (ordered pairs); D (Hermitian) is kept apart
enum JobSq { J_E = 0, J_F, J_GX, J_QV, J_X, J_GZ, NJSQ };   // J_X holds X2 = 2 X
// output terms
enum Term { T_A = 0, T_PHIX, T_PHIY, T_PHIZ, T_PHI, T_XI, T_RES, NTERM };
// one-point statistics per y (FP64 sums over snapshots and the plane)
enum Stat { S_Q = 0, S_UV, S_PV, S_QU, S_QV, S_QW, S_EPS, NSTAT };

template <typename T> struct cplx { T x, y; };
typedef cplx<double> zd;
typedef cplx<float> zf;

template <typename T> __device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return mk(s * a.x, s * a.y); }
template <typename T> __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return mk(a.x, -a.y); }
// multiply by i
template <typename T> __device__ __forceinline__ cplx<T> mul_i(cplx<T> a) { return mk(-a.y, a.x); }

__host__ __device__ __forceinline__ int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

__device__ __forceinline__ int bitrev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

// In-place radix-2 decimation-in-time FFT of `nb` sequences of length n = 2^lg
// stored at buf[b * ld + i], done by the whole thread block.  The data must
// already be in bit-reversed order (use bitrev() when loading).
// tw[m] = exp(-2 pi i m / n), m < n/2 (host-computed); sign = -1 forward, +1
// inverse (the inverse is unnormalised).  Ends with __syncthreads().
template <typename T>
__device__ void fft_radix2_block(cplx<T>* buf, int ld, int nb, int lg, const cplx<T>* __restrict__ tw, int sign)
{
    const int n = 1 << lg;
    const int nh = n >> 1;
    __syncthreads();
    for (int s = 1; s <= lg; ++s) {
        const int half = 1 << (s - 1);
        const int tstride = n >> s;            // twiddle step for this stage
        for (int t = threadIdx.x; t < nb * nh; t += blockDim.x) {
            int b = t / nh, j = t - b * nh;
            int grp = j >> (s - 1), pos = j & (half - 1);
            int i0 = grp * (half << 1) + pos, i1 = i0 + half;
            cplx<T> w = tw[pos * tstride];
            if (sign > 0) w.y = -w.y;
            cplx<T>* p = buf + (size_t)b * ld;
            cplx<T> a = p[i0], c = w * p[i1];
            p[i0] = a + c;
            p[i1] = a - c;
        }
        __syncthreads();
    }
}

// signed wavenumber index of FFT bin m of an n-point transform, 0 at Nyquist
__host__ __device__ __forceinline__ int signed_bin(int m, int n) {
    if (2 * m == n) return 0;
    return (m < n / 2 + (n & 1)) ? m : m - n;
}

__host__ __device__ __forceinline__ long long pair_index(int i1, int i2, int ny) {
    // row-major enumeration of pairs i1 <= i2
    return (long long)i1 * ny - (long long)i1 * (i1 - 1) / 2 + (i2 - i1);
}

}  // namespace gke
