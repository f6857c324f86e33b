// gke_common.cuh -- device helpers shared by the GKE kernels.
//
// Layout conventions of the Parseval path (all device memory, C order):
//   fields   complex128 [nsnap][4][ny][nz][nxh] input Fourier coefficients of
//            u, v, w, p, forward-normalised: a_hat(k) = (1/(nx nz)) sum_x a e^{-ik.x}
//   Xop      complex<TF> [NFIELD][Nk][ns][ny]  correlator operands, one block
//            of ns x ny values per (field, wavenumber); Nk = nz * nxh,
//            k = kz_index * nxh + kx_index; TF = double (plain path) or
//            float (split path)
//   raw      complex [NJOB][YB][YB][Nk][8][8]  one batch's contractions on ordered
//            pairs (y, y') in 8 x 8 blocks, YB = ceil(ny / 8): block (y/8, y'/8),
//            then the wavenumber, then (y % 8, y' % 8) (raw_index; D: only
//            y <= y' is meaningful)
//   comb     complex128 [npair][NTERM][Nk]     per-pair term spectra summed over
//            batches (the FP64 snapshot-sum accumulator)
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
constexpr int J_D = NJSQ;          // Hermitian contraction D, stored after the square jobs
constexpr int NJOB = NJSQ + 1;
// output terms
enum Term { T_A = 0, T_PHIX, T_PHIY, T_PHIZ, T_PHI, T_XI, T_RES, NTERM };
// Spectra written per (plane, wavenumber, pair) by the split correlator's
// plane mode, from which the inverse transforms form the seven terms:
// A; S4 = Gx - Gx^H and S6 = Gz - Gz^H (Phi_x, Phi_z without their D parts);
// Phi_y; phi; xi.  Layout planes[NPLANE][Kc][npp], npp = npair rounded up
// to a multiple of 4 (one wavenumber's values of consecutive pairs are
// contiguous; four pairs fill a 32-byte sector).
enum Plane { PL_A = 0, PL_S4, PL_PHIY, PL_S6, PL_PHI, PL_XI, NPLANE };
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


// One Stockham stage of radix R (2, 3 or 4) with current span Ns over nb
// sequences of length N: butterfly j (< N/R) takes x[j + r N/R] (r < R),
// multiplies by w^(r (j mod Ns) N/(Ns R)), applies the R-point DFT and stores
// to y[(j / Ns) Ns R + (j mod Ns) + r Ns].  cin: conjugate the inputs (first
// stage of an inverse transform).
template <typename T, int R>
__device__ __forceinline__ void fft_stage(const cplx<T>* x, cplx<T>* y, int ld, int nb, int N, int Ns, bool cin,
                                          const cplx<T>* tw)
{
    const int nbf = N / R, tws = N / (Ns * R);
    for (int t = threadIdx.x; t < nb * nbf; t += blockDim.x) {
        const int b = t / nbf, j = t - b * nbf;
        const int jm = j % Ns;
        const cplx<T>* src = x + (size_t)b * ld;
        cplx<T> v[R];
        #pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = src[j + r * nbf];
            if (cin) v[r].y = -v[r].y;
        }
        if (Ns > 1) {
            #pragma unroll
            for (int r = 1; r < R; ++r) v[r] = v[r] * tw[r * jm * tws];
        }
        cplx<T>* dst = y + (size_t)b * ld + (j - jm) * R + jm;
        if (R == 2) {
            dst[0] = v[0] + v[1];
            dst[Ns] = v[0] - v[1];
        } else if (R == 3) {
            // w = e^{-2 pi i/3} = -1/2 - i sqrt(3)/2
            const T h = (T)0.5, s3 = (T)0.86602540378443864676;
            const cplx<T> t1 = v[1] + v[2], t2 = v[1] - v[2];
            const cplx<T> m1 = mk(v[0].x - h * t1.x, v[0].y - h * t1.y);
            const cplx<T> m2 = mk(s3 * t2.y, -s3 * t2.x);          // -i sqrt(3)/2 (v1 - v2)
            dst[0] = v[0] + t1;
            dst[Ns] = m1 + m2;
            dst[2 * Ns] = m1 - m2;
        } else {
            const cplx<T> a0 = v[0] + v[2], a1 = v[0] - v[2], a2 = v[1] + v[3];
            const cplx<T> d = v[1] - v[3];
            const cplx<T> a3 = mk(d.y, -d.x);          // -i (v1 - v3)
            dst[0] = a0 + a2;
            dst[Ns] = a1 + a3;
            dst[2 * Ns] = a0 - a2;
            dst[3 * Ns] = a1 - a3;
        }
    }
}

// Forward transform X[k] = sum_n x[n] e^{-2 pi i n k / N} of nb sequences
// x[b * ld + n], N = 2^a or 3 * 2^a, by the whole thread block: Stockham
// autosort (natural order in and out) with a radix-3 stage when 3 divides N,
// a radix-2 stage when a is odd, then radix-4 stages (fft_stage).
// tw[m] = e^{-2 pi i m / N}, m < N (host-computed, staged in shared memory
// by the caller).  INV = true computes the unnormalised inverse (conjugate
// in, forward transform, conjugate out).  Returns the buffer that holds the
// result (x or y); begins and ends with __syncthreads().
template <typename T, bool INV>
__device__ cplx<T>* fft_block(cplx<T>* x, cplx<T>* y, int ld, int nb, int N, const cplx<T>* tw)
{
    __syncthreads();
    int Ns = 1;
    bool first = true;
    const int p2 = (N % 3 == 0) ? N / 3 : N;      // power-of-two part
    auto swap = [&]() { cplx<T>* tmp = x; x = y; y = tmp; };
    if (p2 != N) {
        fft_stage<T, 3>(x, y, ld, nb, N, Ns, INV && first, tw);
        __syncthreads();
        swap();
        Ns *= 3;
        first = false;
    }
    if (ilog2(p2) & 1) {
        fft_stage<T, 2>(x, y, ld, nb, N, Ns, INV && first, tw);
        __syncthreads();
        swap();
        Ns *= 2;
        first = false;
    }
    while (Ns < N) {
        fft_stage<T, 4>(x, y, ld, nb, N, Ns, INV && first, tw);
        __syncthreads();
        swap();
        Ns *= 4;
        first = false;
    }
    if (INV) {
        for (int t = threadIdx.x; t < nb * N; t += blockDim.x) {
            const int b = t / N, i = t - b * N;
            x[(size_t)b * ld + i].y = -x[(size_t)b * ld + i].y;
        }
        __syncthreads();
    }
    return x;
}

// stage the N-entry twiddle table in shared memory (call before fft_block)
template <typename T>
__device__ __forceinline__ void load_twiddles(cplx<T>* sh_tw, const cplx<T>* __restrict__ tw, int N)
{
    for (int i = threadIdx.x; i < N; i += blockDim.x) sh_tw[i] = tw[i];
}

// ---------------------------------------------------------------- register FFT
// W_32^j = e^{-2 pi i j / 32}, j < 16: values of the host libm cos / sin,
// written out (each translation unit has its own copy)
static __constant__ zd c_tw32d[16] = {
    {1.0, -0.0},
    {0.98078528040323043, -0.19509032201612825},
    {0.92387953251128674, -0.38268343236508978},
    {0.83146961230254524, -0.55557023301960218},
    {0.70710678118654757, -0.70710678118654746},
    {0.55557023301960229, -0.83146961230254524},
    {0.38268343236508984, -0.92387953251128674},
    {0.19509032201612833, -0.98078528040323043},
    {6.123233995736766e-17, -1},
    {-0.19509032201612819, -0.98078528040323043},
    {-0.38268343236508973, -0.92387953251128674},
    {-0.55557023301960196, -0.83146961230254546},
    {-0.70710678118654746, -0.70710678118654757},
    {-0.83146961230254535, -0.55557023301960218},
    {-0.92387953251128674, -0.38268343236508989},
    {-0.98078528040323043, -0.19509032201612861}};
static __constant__ zf c_tw32f[16] = {
    {1.0f, -0.0f},
    {0.98078528f, -0.195090322f},
    {0.923879533f, -0.382683432f},
    {0.831469612f, -0.555570233f},
    {0.707106781f, -0.707106781f},
    {0.555570233f, -0.831469612f},
    {0.382683432f, -0.923879533f},
    {0.195090322f, -0.98078528f},
    {6.123234e-17f, -1.0f},
    {-0.195090322f, -0.98078528f},
    {-0.382683432f, -0.923879533f},
    {-0.555570233f, -0.831469612f},
    {-0.707106781f, -0.707106781f},
    {-0.831469612f, -0.555570233f},
    {-0.923879533f, -0.382683432f},
    {-0.98078528f, -0.195090322f}};
template <typename T> __device__ __forceinline__ cplx<T> tw32(int j);
template <> __device__ __forceinline__ zf tw32<float>(int j) { return c_tw32f[j]; }
template <> __device__ __forceinline__ zd tw32<double>(int j) { return c_tw32d[j]; }

// w * W_32^m (conjugate twiddle if INV) for m known at compile time after
// unrolling: m = 0 and m = 8 (-i) cost no arithmetic, m = 4 and m = 12
// ((+-1 - i)/sqrt 2) two additions and two multiplications
template <typename T, bool INV>
__device__ __forceinline__ cplx<T> twiddle_mul(cplx<T> w, int m)
{
    const T c = (T)0.70710678118654752440;
    if (m == 0) return w;
    if (m == 8) return INV ? mk(-w.y, w.x) : mk(w.y, -w.x);
    if (m == 4) return INV ? mk(c * (w.x - w.y), c * (w.x + w.y)) : mk(c * (w.x + w.y), c * (w.y - w.x));
    if (m == 12) return INV ? mk(-c * (w.x + w.y), c * (w.x - w.y)) : mk(c * (w.y - w.x), -c * (w.x + w.y));
    cplx<T> t = tw32<T>(m);
    if (INV) t.y = -t.y;
    return w * t;
}

template <int M> struct Lg2 { static constexpr int v = Lg2<M / 2>::v + 1; };
template <> struct Lg2<1> { static constexpr int v = 0; };
__host__ __device__ constexpr int brev_ct(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r = (r << 1) | ((x >> i) & 1);
    return r;
}

// butterflies of span LEN of the radix-2 DFT in registers (LEN a template
// parameter, so every twiddle index is a compile-time constant), then LEN * 2
template <typename T, int M, int LEN, bool INV>
__device__ __forceinline__ void dft_stage(cplx<T>* a)
{
    #pragma unroll
    for (int i = 0; i < M; i += LEN) {
        #pragma unroll
        for (int j = 0; j < LEN / 2; ++j) {
            const cplx<T> u = a[i + j], w = twiddle_mul<T, INV>(a[i + j + LEN / 2], j * (32 / LEN));
            a[i + j] = u + w;
            a[i + j + LEN / 2] = u - w;
        }
    }
    if constexpr (LEN < M) dft_stage<T, M, 2 * LEN, INV>(a);
}

// M-point DFT (M <= 32, power of two) of v[0..M) in registers, natural order in
// and out: radix-2 decimation in time on the bit-reversed copy; INV conjugates
// the twiddles (unnormalised inverse).
template <typename T, int M, bool INV>
__device__ __forceinline__ void dft_reg(cplx<T>* v)
{
    cplx<T> a[M];
    #pragma unroll
    for (int i = 0; i < M; ++i) a[brev_ct(i, Lg2<M>::v)] = v[i];
    dft_stage<T, M, 2, INV>(a);
    #pragma unroll
    for (int i = 0; i < M; ++i) v[i] = a[i];
}

// Two-level transform of one sequence of N = N1 N2 points held by N2 lanes:
// on entry lane n2 holds v[m] = x[n2 + N2 m] (m < N1); on exit v[m] =
// X[n2 + N2 m], X[k] = sum_n x[n] w^{n k} (w = e^{-2 pi i / N}, conjugate if
// INV, unnormalised).  n = N2 n1 + n2, k = k1 + N1 k2:
//   X[k1 + N1 k2] = sum_n2 W_N2^{n2 k2} [ w^{n2 k1} sum_n1 x[N2 n1 + n2] W_N1^{n1 k1} ].
// The inner DFT runs in registers, its twiddled result goes through the
// exchange buffer xs[k1 s1 + n2 s2] and the outer DFT (rows k1 = n2 + N2 j)
// runs in registers again.  stw: the N-point twiddle table in shared memory.
// Contains one __syncthreads(); every thread of the block must call it.
template <typename T, int N1, int N2, bool INV>
__device__ __forceinline__ void fft2l(cplx<T>* v, int lane, cplx<T>* xs, int s1, int s2, const cplx<T>* stw)
{
    static_assert(N1 % N2 == 0, "N1 must be a multiple of N2");
    constexpr int R = N1 / N2;
    dft_reg<T, N1, INV>(v);
    #pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) {
        cplx<T> w = stw[lane * k1];
        if (INV) w.y = -w.y;
        v[k1] = v[k1] * w;
    }
    #pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) xs[k1 * s1 + lane * s2] = v[k1];
    __syncthreads();
    #pragma unroll
    for (int jj = 0; jj < R; ++jj) {
        const int k1 = lane + N2 * jj;
        cplx<T> b[N2];
        #pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) b[n2] = xs[k1 * s1 + n2 * s2];
        dft_reg<T, N2, INV>(b);
        #pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[jj + R * k2] = b[k2];     // X[lane + N2 (jj + R k2)]
    }
}

// streaming (evict-first) loads and stores for data touched once, so that
// they do not push reused working sets out of L2
__device__ __forceinline__ cplx<float> ld_stream(const cplx<float>* p) {
    const float2 v = __ldcs((const float2*)p);
    cplx<float> r; r.x = v.x; r.y = v.y; return r;
}
__device__ __forceinline__ cplx<double> ld_stream(const cplx<double>* p) {
    const double2 v = __ldcs((const double2*)p);
    cplx<double> r; r.x = v.x; r.y = v.y; return r;
}
__device__ __forceinline__ void st_stream(cplx<float>* p, cplx<float> v) { __stcs((float2*)p, make_float2(v.x, v.y)); }
__device__ __forceinline__ void st_stream(cplx<double>* p, cplx<double> v) {
    __stcs((double2*)p, make_double2(v.x, v.y));
}
__device__ __forceinline__ void st_stream(float* p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(double* p, double v) { __stcs(p, v); }

// signed wavenumber index of FFT bin m of an n-point transform, 0 at Nyquist
__host__ __device__ __forceinline__ int signed_bin(int m, int n) {
    if (2 * m == n) return 0;
    return (m < n / 2 + (n & 1)) ? m : m - n;
}

__host__ __device__ __forceinline__ long long raw_index(int job, long long k, int y, int yp, int Nk, int YB) {
    return ((((long long)job * YB + (y >> 3)) * YB + (yp >> 3)) * Nk + k) * 64 + ((y & 7) << 3) + (yp & 7);
}

__host__ __device__ __forceinline__ long long pair_index(int i1, int i2, int ny) {
    // row-major enumeration of pairs i1 <= i2
    return (long long)i1 * ny - (long long)i1 * (i1 - 1) / 2 + (i2 - i1);
}

__host__ __device__ __forceinline__ long long wedge_index(int i1, int i2, int ny) {
    // row-major enumeration of the half-channel wedge i1 <= i2, i1 + i2 <= ny - 1
    return (long long)i1 * ny - (long long)i1 * (i1 - 1) + (i2 - i1);
}

// Where the value of a term at the ordered pair (a, b) is stored: the pair
// index, the sign and whether the separation is inverted (r -> -r).  Pairs
// below the diagonal come from r-inversion, (a, b, r) -> (b, a, -r), parity
// rho (Sec. 3.3); on the wedge, pairs past the anti-diagonal a + b = ny - 1
// come from the combined inversion of y and r, (a, b, r) -> (ny-1-b, ny-1-a,
// -r), parity sigma.
template <typename T>
__host__ __device__ __forceinline__ long long stored_pair(int a, int b, int ny, bool wedge, T rho, T sigma,
                                                          T& sg, bool& flip)
{
    sg = (T)1;
    flip = false;
    if (a > b) { const int t = a; a = b; b = t; sg *= rho; flip = !flip; }
    if (wedge && a + b > ny - 1) {
        const int na = ny - 1 - b, nb = ny - 1 - a;
        a = na; b = nb;
        sg *= sigma;
        flip = !flip;
    }
    return wedge ? wedge_index(a, b, ny) : pair_index(a, b, ny);
}

}  // namespace gke
