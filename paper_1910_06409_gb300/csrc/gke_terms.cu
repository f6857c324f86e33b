// gke_terms.cu -- from per-pair term spectra to the GKE terms.
//
// Inverse transform (Sec. 3.1, Eq. 9) of the term spectra comb[p][t][k]
// (formed by k_combine), the one-point parts of the correlation expansion
// (Eq. 7), and the Step-3 finite-difference derivatives in Y1 / Y2
// (Sec. 3.2, Eq. 10-11) with values across the diagonal recovered by
// r-inversion (Sec. 3.3).  One-point parts, with q = u_i u_i:
//   A     : <q>1 + <q>2
//   Phi_x : <qu>2 - <qu>1 + dU (<q>1 + <q>2)
//   Phi_y : <qv>2 - <qv>1                                   (+ FD part)
//   Phi_z : <qw>2 - <qw>1
//   phi   : (<qv>1 + <qv>2)/2 + 2 (<pv>1 + <pv>2)          (+ FD part)
//   xi    : -2 U'* (<uv>1 + <uv>2) - dU' (<uv>2 - <uv>1) - 2 (eps1 + eps2)
//   res   : -xi                                             (+ FD parts)
//
// Plain path: transforms, terms and stencils in FP64.  Split path:
// transforms in FP32 and FP32 terms; the Step-3 stencils difference the
// spectral part of each term (kept apart in FP32 scratch) in FP32 and the
// one-point part, a function of (Y1, Y2) only, in FP64 once per pair, so the
// large one-point values never pass through an FP32 difference.
#include "gke_common.cuh"
#include "gke_kernels.h"

namespace gke {

// -------------------------- column pass: inverse transform along z
// W[pl][t][z][kx] = sum_kz comb[p][t][kz, kx] e^{+i kz z} (the 1/count of the
// average is applied by the row pass, with the one-point parts).
// CTA = CW kx columns of one term of one pair; shared memory (1 + 2 CW) nz
// complex.
template <typename TF, typename TB>
__global__ void k_terms_colpass(const cplx<TB>* __restrict__ comb, long long pair0, int nz, int nx, int CW,
                                const cplx<TF>* __restrict__ tw_z, SepMap sm, unsigned tmask,
                                cplx<TF>* __restrict__ W)
{
    typedef cplx<TF> C;
    extern __shared__ __align__(16) unsigned char sh_raw_tc[];
    C* stw = (C*)sh_raw_tc;
    C* b0 = stw + nz;
    C* b1 = b0 + CW * nz;
    const int nxh = nx / 2 + 1, Nk = nz * nxh;
    const int kx0 = blockIdx.x * CW, q = nth_bit(tmask, blockIdx.y);     // grid.y: the terms of tmask
    const long long pl = blockIdx.z, p = pair0 + pl;
    load_twiddles(stw, tw_z, nz);
    const cplx<TB>* src = comb + (p * NTERM + q) * (long long)Nk;
    for (int t = threadIdx.x; t < CW * nz; t += blockDim.x) {
        const int c = t % CW, kz_i = t / CW, kx_i = kx0 + c;
        C v = mk((TF)0, (TF)0);
        if (kx_i < nxh) {
            const cplx<TB> x = src[(long long)kz_i * nxh + kx_i];
            v = mk((TF)x.x, (TF)x.y);
        }
        b0[c * nz + kz_i] = v;
    }
    const C* res = fft_block<TF, true>(b0, b1, nz, CW, nz, stw);
    C* dst = W + (pl * NTERM + q) * (long long)sm.nrz * nxh;
    for (int t = threadIdx.x; t < CW * nz; t += blockDim.x) {
        const int c = t % CW, z = t / CW, kx_i = kx0 + c;
        const int zr = sm.zrow(z);
        if (kx_i < nxh && zr >= 0) dst[(long long)zr * nxh + kx_i] = res[c * nz + z];
    }
}

// register-FFT column pass for nz = N1 N2: CTA = CW columns of one term of
// one pair x N2 lanes (see fft2l)
template <typename TF, typename TB, int N1, int N2, bool US>
__global__ void __launch_bounds__(256)
k_terms_colpass_r(const cplx<TB>* __restrict__ comb, long long pair0, int nxh, int CW,
                  const cplx<TF>* __restrict__ tw_z, SepMap sm, unsigned tmask, cplx<TF>* __restrict__ W)
{
    typedef cplx<TF> C;
    constexpr int N = N1 * N2;
    extern __shared__ __align__(16) unsigned char sh_raw_tcr[];
    C* stw = (C*)sh_raw_tcr;
    C* xs = stw + N;
    const int c = threadIdx.x % CW, lane = threadIdx.x / CW;
    const int kx = blockIdx.x * CW + c, q = nth_bit(tmask, blockIdx.y);
    const long long pl = blockIdx.z, p = pair0 + pl;
    const int Nk = N * nxh;
    load_twiddles(stw, tw_z, N);
    const cplx<TB>* src = comb + (p * NTERM + q) * (long long)Nk;
    C v[N1];
    #pragma unroll
    for (int m = 0; m < N1; ++m) {
        C x = mk((TF)0, (TF)0);
        if (kx < nxh) {
            const cplx<TB> b = ld_stream(src + (long long)(lane + N2 * m) * nxh + kx);
            x = mk((TF)b.x, (TF)b.y);
        }
        v[m] = x;
    }
    __syncthreads();
    fft2l<TF, N1, N2, true>(v, lane, xs + c, N2 * CW + 1, CW, stw);
    if (kx < nxh) {
        C* dst = W + (pl * NTERM + q) * (long long)(US ? sm.nrz : N) * nxh;
        #pragma unroll
        for (int m = 0; m < N1; ++m) {
            const int zr = US ? sm.zrow(lane + N2 * m) : lane + N2 * m;
            if (zr >= 0) dst[(long long)zr * nxh + kx] = v[m];
        }
    }
}

// one-point parts of the seven terms at the pair (i1, i2), FP64
__device__ __forceinline__ void onepoint(const double* __restrict__ pr, int ny, int i1, int i2, double one[NTERM])
{
    const double q1 = pr[PR_Q * ny + i1], q2 = pr[PR_Q * ny + i2];
    const double uv1 = pr[PR_UV * ny + i1], uv2 = pr[PR_UV * ny + i2];
    const double pv1 = pr[PR_PV * ny + i1], pv2 = pr[PR_PV * ny + i2];
    const double qu1 = pr[PR_QU * ny + i1], qu2 = pr[PR_QU * ny + i2];
    const double qv1 = pr[PR_QV * ny + i1], qv2 = pr[PR_QV * ny + i2];
    const double qw1 = pr[PR_QW * ny + i1], qw2 = pr[PR_QW * ny + i2];
    const double e1 = pr[PR_EPS * ny + i1], e2 = pr[PR_EPS * ny + i2];
    const double dU = pr[PR_U * ny + i2] - pr[PR_U * ny + i1];
    const double Upm = 0.5 * (pr[PR_DU * ny + i1] + pr[PR_DU * ny + i2]);
    const double dUp = pr[PR_DU * ny + i2] - pr[PR_DU * ny + i1];
    one[T_A] = q1 + q2;
    one[T_PHIX] = (qu2 - qu1) + dU * (q1 + q2);
    one[T_PHIY] = qv2 - qv1;
    one[T_PHIZ] = qw2 - qw1;
    one[T_PHI] = 0.5 * (qv1 + qv2) + 2.0 * (pv1 + pv2);
    one[T_XI] = -2.0 * Upm * (uv1 + uv2) - dUp * (uv2 - uv1) - 2.0 * (e1 + e2);
    one[T_RES] = -one[T_XI];
}

// ------------------------------ row pass: C2R along x + one-point parts
// terms[t][p][z][x] = inv_count sum_kx W[pl][t][z][kx] e^{+i kx x} + onepoint_t(Y1, Y2),
// stored as TO.  With spec != NULL (the FP32 path) the spectral parts of A,
// Phi_y and phi (the terms the Step-3 stencils difference) go to
// spec[3][p][z][x], and Phi_y and phi go there only: the first stencil pass
// writes those two terms.
// Terms are transformed two at a time (t0 + i t1).  CTA = RZ rows of one pair;
// shared memory (1 + 8 RZ) nx complex.
template <typename TF, typename TO>
__global__ void k_terms_rowpass(const cplx<TF>* __restrict__ W, const int* __restrict__ pair_i, long long pair0,
                                long long npair, int ny, int nx, int RZ, double inv_count,
                                const double* __restrict__ prof, const cplx<TF>* __restrict__ tw_x, SepMap sm,
                                unsigned tmask, TO* __restrict__ terms, float* __restrict__ spec)
{
    typedef cplx<TF> C;
    extern __shared__ __align__(16) unsigned char sh_raw_tr[];
    C* stw = (C*)sh_raw_tr;
    C* b0 = stw + nx;
    C* b1 = b0 + RZ * 4 * nx;
    __shared__ TF s_one[NTERM];
    const int nxh = nx / 2 + 1;
    const int nz = sm.nrz;                 // rows kept (all nz at full resolution)
    const int z0 = blockIdx.x * RZ;
    const int nrow = min(RZ, nz - z0);
    const long long pl = blockIdx.y, p = pair0 + pl;
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    load_twiddles(stw, tw_x, nx);
    if (threadIdx.x == 0) {
        double one[NTERM];
        onepoint(prof, ny, i1, i2, one);
        for (int t = 0; t < NTERM; ++t) s_one[t] = (TF)one[t];
    }
    for (int t = threadIdx.x; t < nrow * 4 * nx; t += blockDim.x) {
        int r = t / (4 * nx), rem = t - r * 4 * nx, j = rem / nx, k = rem - j * nx;
        int z = z0 + r;
        int ta = 2 * j, tb = 2 * j + 1;
        const C* wa = W + ((pl * NTERM + ta) * nz + z) * nxh;
        C A = mk((TF)0, (TF)0), B = A;               // terms outside tmask: zero, not stale W
        if ((tmask >> ta) & 1u) { if (k < nxh) A = wa[k]; else A = conj(wa[nx - k]); }
        if (tb < NTERM && ((tmask >> tb) & 1u)) {
            const C* wb = W + ((pl * NTERM + tb) * nz + z) * nxh;
            if (k < nxh) B = wb[k]; else B = conj(wb[nx - k]);
        }
        if (k == 0 || 2 * k == nx) { A.y = 0; B.y = 0; }
        b0[(r * 4 + j) * nx + k] = mk(A.x - B.y, A.y + B.x);
    }
    const C* sh = fft_block<TF, true>(b0, b1, nx, 4 * nrow, nx, stw);
    const long long N = (long long)nz * sm.nrx;
    for (int t = threadIdx.x; t < nrow * NTERM * nx; t += blockDim.x) {
        int r = t / (NTERM * nx), rem = t - r * NTERM * nx, q = rem / nx, x = rem - q * nx;
        const int xr = sm.xcol(x);
        if (xr < 0 || !((tmask >> q) & 1u)) continue;
        C v = sh[(r * 4 + (q >> 1)) * nx + x];
        const TF sp = ((q & 1) ? v.y : v.x) * (TF)inv_count;
        const long long e = (long long)(z0 + r) * sm.nrx + xr;
        if (spec == nullptr || (q != T_PHIY && q != T_PHI)) terms[((long long)q * npair + p) * N + e] = (TO)(sp + s_one[q]);
        if (spec != nullptr) {
            const int si = (q == T_A) ? 0 : (q == T_PHIY) ? 1 : (q == T_PHI) ? 2 : -1;
            if (si >= 0) spec[((long long)si * npair + p) * N + e] = (float)sp;
        }
    }
}

// register-FFT row pass for nx = N1 N2: CTA = RZ rows of one pair x N2 lanes;
// the seven terms are transformed as four packed sequences (t0 + i t1, ...)
template <typename TF, typename TO, int N1, int N2, bool US>
__global__ void __launch_bounds__(256)
k_terms_rowpass_r(const cplx<TF>* __restrict__ W, const int* __restrict__ pair_i, long long pair0, long long npair,
                  int ny, int RZ, double inv_count, const double* __restrict__ prof,
                  const cplx<TF>* __restrict__ tw_x, SepMap sm, unsigned tmask, TO* __restrict__ terms,
                  float* __restrict__ spec)
{
    typedef cplx<TF> C;
    constexpr int N = N1 * N2, nxh = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char sh_raw_trr[];
    C* stw = (C*)sh_raw_trr;
    C* xs = stw + N;
    __shared__ TF s_one[NTERM];
    const int lane = threadIdx.x % N2, r = threadIdx.x / N2;
    const int nz = sm.nrz;                 // rows kept (all nz at full resolution)
    const int nrx = US ? sm.nrx : N;
    const int z = blockIdx.x * RZ + r;
    const bool live = z < nz;
    const long long pl = blockIdx.y, p = pair0 + pl;
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    load_twiddles(stw, tw_x, N);
    if (threadIdx.x == 0) {
        double one[NTERM];
        onepoint(prof, ny, i1, i2, one);
        for (int t = 0; t < NTERM; ++t) s_one[t] = (TF)one[t];
    }
    const long long NN = (long long)nz * nrx;
    const TF ic = (TF)inv_count;
    C* xr = xs + r * N1 * (N2 + 1);
    for (int jq = 0; jq < 4; ++jq) {
        const int ta = 2 * jq, tb = 2 * jq + 1;
        const bool ha = (tmask >> ta) & 1u, hb = tb < NTERM && ((tmask >> tb) & 1u);
        if (!ha && !hb) continue;                   // uniform over the CTA
        const C* wa = W + ((pl * NTERM + ta) * nz + (live ? z : 0)) * nxh;
        const C* wb = W + ((pl * NTERM + (tb < NTERM ? tb : ta)) * nz + (live ? z : 0)) * nxh;
        C v[N1];
        #pragma unroll
        for (int m = 0; m < N1; ++m) {
            const int k = lane + N2 * m;
            C A = mk((TF)0, (TF)0), B = A;           // terms outside tmask: zero, not stale W
            if (ha) { if (k < nxh) A = wa[k]; else A = conj(wa[N - k]); }
            if (hb) { if (k < nxh) B = wb[k]; else B = conj(wb[N - k]); }
            if (k == 0 || 2 * k == N) { A.y = 0; B.y = 0; }
            v[m] = mk(A.x - B.y, A.y + B.x);
        }
        __syncthreads();                     // exchange buffer free (and s_one, twiddles ready)
        fft2l<TF, N1, N2, true>(v, lane, xr, N2 + 1, 1, stw);
        if (live) {
            #pragma unroll
            for (int m = 0; m < N1; ++m) {
                const int xr = US ? sm.xcol(lane + N2 * m) : lane + N2 * m;
                if (xr < 0) continue;
                const long long e = (long long)z * nrx + xr;
                #pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = 2 * jq + h;
                    if (q >= NTERM) break;
                    if (!(h ? hb : ha)) continue;
                    const TF sp = (h ? v[m].y : v[m].x) * ic;
                    if (spec == nullptr || (q != T_PHIY && q != T_PHI))
                        st_stream(terms + ((long long)q * npair + p) * NN + e, (TO)(sp + s_one[q]));
                    if (spec != nullptr) {
                        const int si = (q == T_A) ? 0 : (q == T_PHIY) ? 1 : (q == T_PHI) ? 2 : -1;
                        if (si >= 0) st_stream(spec + ((long long)si * npair + p) * NN + e, (float)sp);
                    }
                }
            }
        }
    }
}

// ------------------- column pass from the plane spectra (split plane mode)
// The seven term spectra of a pair at wavenumber (kz, kx) from its planes
// (Sec. 3.1, Eq. 7 grouped by term; the D parts of Phi_x, Phi_z and the
// residual, whose coefficients depend on the pair and the wavenumber only,
// are added here):
//   A, Phi_x = S4 + (dU - 2 i nu kx) A, Phi_y, Phi_z = S6 - 2 i nu kz A, phi,
//   xi, res = i kx Phi_x + i kz Phi_z - xi         (dU = U(Y2) - U(Y1)),
// then the inverse transform along z into W, as k_terms_colpass.
// Column (pair, kx): a CTA takes 4 kx of one group of 4 pairs, so the loads
// of one kz row are four whole 32-byte sectors of the planes.
// a cached load the compiler keeps in program order (not hoisted out of
// the term loop, where it would hold a whole column in registers)
__device__ __forceinline__ cplx<float> ld_ordered(const cplx<float>* p)
{
    cplx<float> r;
    asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ cplx<double> ld_ordered(const cplx<double>* p)
{
    cplx<double> r;
    asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
    return r;
}

struct PlaneCols {
    const void* planes; long long npp; int Kc;
    const int* pair_i; const double* prof; int ny; double Lx, Lz, nu;
};

// register variant, nz = N1 N2: CTA = 16 columns x N2 lanes; all terms of
// tmask (and those the residual is formed from) in one CTA
template <typename TF, typename TB, int N1, int N2, bool US>
__global__ void __launch_bounds__(256, 2)
k_terms_colpass_planes_r(PlaneCols pc, long long pair0, long long npair, int nx, const cplx<TF>* __restrict__ tw_z,
                         SepMap sm, unsigned tmask, cplx<TF>* __restrict__ W)
{
    typedef cplx<TF> C;
    constexpr int N = N1 * N2, CW = 16;
    extern __shared__ __align__(16) unsigned char sh_raw_tpr[];
    C* stw = (C*)sh_raw_tpr;
    C* xs = stw + N;
    const int c = threadIdx.x % CW, lane = threadIdx.x / CW;
    const int q4 = c & 3, nxh = nx / 2 + 1;
    // grid.x: pair groups (consecutive CTAs read adjacent sectors), grid.y: kx groups
    const int kx = blockIdx.y * 4 + (c >> 2);
    const long long g = pair0 / 4 + blockIdx.x;
    const long long p = 4 * g + q4, pl = p - pair0;
    const bool live = kx < nxh && p < npair;
    load_twiddles(stw, tw_z, N);
    TF dU = 0, kxv = 0;
    if (live) {
        const int i1 = pc.pair_i[2 * p], i2 = pc.pair_i[2 * p + 1];
        dU = (TF)(pc.prof[PR_U * pc.ny + i2] - pc.prof[PR_U * pc.ny + i1]);
        kxv = (TF)(6.283185307179586476925286766559 * signed_bin(kx, nx) / pc.Lx);
    }
    const TF nu2 = (TF)(2.0 * pc.nu), kzs = (TF)(6.283185307179586476925286766559 / pc.Lz);
    const cplx<TB>* base = (const cplx<TB>*)pc.planes + (long long)kx * pc.npp + p;
    const long long pstride = (long long)pc.Kc * pc.npp, kzs_el = (long long)nxh * pc.npp;
    // the planes are read once (streaming loads), except A, which up to three
    // terms use and which is re-read through the caches; each column is
    // walked with a pointer that steps N2 kz rows
    const long long step = (long long)N2 * kzs_el;
    const cplx<TB>* col0 = base + lane * kzs_el;
    auto cv = [](cplx<TB> b) { return mk((TF)b.x, (TF)b.y); };
    const bool want_res = (tmask >> T_RES) & 1u;
    C r[N1], v[N1];
    #pragma unroll
    for (int m = 0; m < N1; ++m) r[m] = mk((TF)0, (TF)0);
    C* dst0 = W + pl * NTERM * (long long)(US ? sm.nrz : N) * nxh;
    #pragma unroll 1
    for (int t = 0; t < NTERM; ++t) {
        const bool out = (tmask >> t) & 1u;
        if (!out && !(want_res && (t == T_PHIX || t == T_PHIZ || t == T_XI))) continue;   // uniform
        if (!live) {
            #pragma unroll
            for (int m = 0; m < N1; ++m) v[m] = mk((TF)0, (TF)0);
        } else if (t == T_A) {
            const cplx<TB>* pa = col0 + PL_A * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, pa += step) v[m] = cv(ld_ordered(pa));
        } else if (t == T_PHIX) {
            const cplx<TB>* ps = col0 + PL_S4 * pstride;
            const cplx<TB>* pa = col0 + PL_A * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, ps += step, pa += step) {
                const C s = cv(ld_stream(ps)), av = cv(ld_ordered(pa));
                v[m] = mk(s.x + dU * av.x + nu2 * kxv * av.y, s.y + dU * av.y - nu2 * kxv * av.x);
                r[m] = mk(r[m].x - kxv * v[m].y, r[m].y + kxv * v[m].x);
            }
        } else if (t == T_PHIZ) {
            const cplx<TB>* ps = col0 + PL_S6 * pstride;
            const cplx<TB>* pa = col0 + PL_A * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, ps += step, pa += step) {
                const C s = cv(ld_stream(ps)), av = cv(ld_ordered(pa));
                const TF kzv = kzs * (TF)signed_bin(lane + N2 * m, N);
                v[m] = mk(s.x + nu2 * kzv * av.y, s.y - nu2 * kzv * av.x);
                r[m] = mk(r[m].x - kzv * v[m].y, r[m].y + kzv * v[m].x);
            }
        } else if (t == T_XI) {
            const cplx<TB>* px = col0 + PL_XI * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, px += step) {
                v[m] = cv(ld_stream(px));
                r[m] = r[m] - v[m];
            }
        } else if (t == T_RES) {
            #pragma unroll
            for (int m = 0; m < N1; ++m) v[m] = r[m];
        } else {
            const cplx<TB>* pj = col0 + (t == T_PHIY ? PL_PHIY : PL_PHI) * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, pj += step) v[m] = cv(ld_stream(pj));
        }
        if (!out) continue;
        __syncthreads();                     // exchange buffer free (twiddles ready)
        fft2l<TF, N1, N2, true>(v, lane, xs + c, N2 * CW + 1, CW, stw);
        if (live) {
            C* dst = dst0 + (long long)t * (US ? sm.nrz : N) * nxh;
            #pragma unroll
            for (int m = 0; m < N1; ++m) {
                const int zr = US ? sm.zrow(lane + N2 * m) : lane + N2 * m;
                if (zr >= 0) dst[(long long)zr * nxh + kx] = v[m];
            }
        }
    }
}

// shared-memory variant, any nz: CTA = 4 KXC columns (KXC kx of one pair group)
template <typename TF, typename TB>
__global__ void k_terms_colpass_planes(PlaneCols pc, long long pair0, long long npair, int nz, int nx, int KXC,
                                       const cplx<TF>* __restrict__ tw_z, SepMap sm, unsigned tmask,
                                       cplx<TF>* __restrict__ W)
{
    typedef cplx<TF> C;
    extern __shared__ __align__(16) unsigned char sh_raw_tp[];
    const int NC = 4 * KXC, nxh = nx / 2 + 1;
    C* stw = (C*)sh_raw_tp;
    C* b0 = stw + nz;
    C* b1 = b0 + NC * nz;
    C* rb = b1 + NC * nz;                     // residual spectrum of each column
    __shared__ TF s_dU[64], s_kx[64];
    const long long g = pair0 / 4 + blockIdx.x;             // grid.x: pair groups, grid.y: kx groups
    load_twiddles(stw, tw_z, nz);
    for (int c = threadIdx.x; c < NC; c += blockDim.x) {
        const long long p = 4 * g + (c & 3);
        const int kx = blockIdx.y * KXC + (c >> 2);
        TF dU = 0;
        if (p < npair) {
            const int i1 = pc.pair_i[2 * p], i2 = pc.pair_i[2 * p + 1];
            dU = (TF)(pc.prof[PR_U * pc.ny + i2] - pc.prof[PR_U * pc.ny + i1]);
        }
        s_dU[c] = dU;
        s_kx[c] = kx < nxh ? (TF)(6.283185307179586476925286766559 * signed_bin(kx, nx) / pc.Lx) : (TF)0;
    }
    for (int e = threadIdx.x; e < NC * nz; e += blockDim.x) rb[e] = mk((TF)0, (TF)0);
    __syncthreads();
    const TF nu2 = (TF)(2.0 * pc.nu);
    const long long pstride = (long long)pc.Kc * pc.npp;
    const bool want_res = (tmask >> T_RES) & 1u;
    for (int t = 0; t < NTERM; ++t) {
        const bool out = (tmask >> t) & 1u;
        if (!out && !(want_res && (t == T_PHIX || t == T_PHIZ || t == T_XI))) continue;   // uniform
        __syncthreads();
        for (int e = threadIdx.x; e < NC * nz; e += blockDim.x) {
            const int c = e % NC, kz = e / NC;
            const long long p = 4 * g + (c & 3);
            const int kx = blockIdx.y * KXC + (c >> 2);
            C v = mk((TF)0, (TF)0);
            if (kx < nxh && p < npair) {
                const cplx<TB>* src = (const cplx<TB>*)pc.planes + ((long long)kz * nxh + kx) * pc.npp + p;
                auto ld = [&](int j) { const cplx<TB> b = src[j * pstride]; return mk((TF)b.x, (TF)b.y); };
                C& r = rb[c * nz + kz];
                if (t == T_A) v = ld(PL_A);
                else if (t == T_PHIX) {
                    const C s = ld(PL_S4), av = ld(PL_A);
                    const TF kxv = s_kx[c];
                    v = mk(s.x + s_dU[c] * av.x + nu2 * kxv * av.y, s.y + s_dU[c] * av.y - nu2 * kxv * av.x);
                    r = mk(r.x - kxv * v.y, r.y + kxv * v.x);
                } else if (t == T_PHIZ) {
                    const C s = ld(PL_S6), av = ld(PL_A);
                    const TF kzv = (TF)(6.283185307179586476925286766559 * signed_bin(kz, nz) / pc.Lz);
                    v = mk(s.x + nu2 * kzv * av.y, s.y - nu2 * kzv * av.x);
                    r = mk(r.x - kzv * v.y, r.y + kzv * v.x);
                } else if (t == T_XI) {
                    v = ld(PL_XI);
                    r = r - v;
                } else if (t == T_RES) v = r;
                else v = ld(t == T_PHIY ? PL_PHIY : PL_PHI);
            }
            b0[c * nz + kz] = v;
        }
        if (!out) continue;
        const C* res = fft_block<TF, true>(b0, b1, nz, NC, nz, stw);
        for (int e = threadIdx.x; e < NC * nz; e += blockDim.x) {
            const int c = e % NC, z = e / NC;
            const long long p = 4 * g + (c & 3);
            const int kx = blockIdx.y * KXC + (c >> 2);
            const int zr = sm.zrow(z);
            if (kx < nxh && p < npair && zr >= 0)
                W[((p - pair0) * NTERM + t) * (long long)sm.nrz * nxh + (long long)zr * nxh + kx] = res[c * nz + z];
        }
    }
}

// columns of the shared-memory variant: 4 kx per CTA while its buffers fit
static int planes_kxc(int nz, size_t csz)
{
    int kxc = 4;
    while (kxc > 1 && (size_t)(1 + 3 * 4 * kxc) * nz * csz > 160 * 1024) kxc /= 2;
    return kxc;
}

// ---------- plane mode at nz = nx = N1 N2: pair-contiguous W between the passes
// The planes hold, per wavenumber, consecutive pairs contiguously, so both
// passes take 16 consecutive pairs per CTA: the column pass reads one
// 128-byte line per (plane, kz) and writes Wp[t][zr][kx][pl] (16 pairs = one
// line per (term, z, kx)); the row pass reads those lines back and stages
// its outputs in shared memory, so each pair's row of separations leaves as
// one contiguous store.  pc = pairs per chunk (the stride of Wp's rows).
template <typename TF, typename TB, int N1, int N2, bool US>
__global__ void __launch_bounds__(256, 2)
k_terms_colpass_pt(PlaneCols pc, long long pair0, long long npair, long long pchunk, int nx,
                   const cplx<TF>* __restrict__ tw_z, SepMap sm, unsigned tmask, cplx<TF>* __restrict__ W)
{
    typedef cplx<TF> C;
    constexpr int N = N1 * N2, CW = 16;
    extern __shared__ __align__(16) unsigned char sh_raw_cpt[];
    C* stw = (C*)sh_raw_cpt;
    C* xs = stw + N;
    const int c = threadIdx.x % CW, lane = threadIdx.x / CW;
    const int nxh = nx / 2 + 1;
    const int kx = blockIdx.y;
    const long long pl = (long long)blockIdx.x * CW + c, p = pair0 + pl;
    const bool live = p < npair && pl < pchunk;
    load_twiddles(stw, tw_z, N);
    TF dU = 0;
    if (live) {
        const int i1 = pc.pair_i[2 * p], i2 = pc.pair_i[2 * p + 1];
        dU = (TF)(pc.prof[PR_U * pc.ny + i2] - pc.prof[PR_U * pc.ny + i1]);
    }
    const TF kxv = (TF)(6.283185307179586476925286766559 * signed_bin(kx, nx) / pc.Lx);
    const TF nu2 = (TF)(2.0 * pc.nu), kzs = (TF)(6.283185307179586476925286766559 / pc.Lz);
    const long long kzs_el = (long long)nxh * pc.npp, pstride = (long long)pc.Kc * pc.npp;
    const long long step = (long long)N2 * kzs_el;
    const cplx<TB>* col0 = (const cplx<TB>*)pc.planes + (long long)kx * pc.npp + p + lane * kzs_el;
    auto cv = [](cplx<TB> b) { return mk((TF)b.x, (TF)b.y); };
    const bool want_res = (tmask >> T_RES) & 1u;
    C r[N1], v[N1];
    #pragma unroll
    for (int m = 0; m < N1; ++m) r[m] = mk((TF)0, (TF)0);
    const int nrz = US ? sm.nrz : N;
    #pragma unroll 1
    for (int t = 0; t < NTERM; ++t) {
        const bool out = (tmask >> t) & 1u;
        if (!out && !(want_res && (t == T_PHIX || t == T_PHIZ || t == T_XI))) continue;   // uniform
        if (!live) {
            #pragma unroll
            for (int m = 0; m < N1; ++m) v[m] = mk((TF)0, (TF)0);
        } else if (t == T_A) {
            const cplx<TB>* pa = col0 + PL_A * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, pa += step) v[m] = cv(ld_ordered(pa));
        } else if (t == T_PHIX) {
            const cplx<TB>* ps = col0 + PL_S4 * pstride;
            const cplx<TB>* pa = col0 + PL_A * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, ps += step, pa += step) {
                const C s = cv(ld_stream(ps)), av = cv(ld_ordered(pa));
                v[m] = mk(s.x + dU * av.x + nu2 * kxv * av.y, s.y + dU * av.y - nu2 * kxv * av.x);
                r[m] = mk(r[m].x - kxv * v[m].y, r[m].y + kxv * v[m].x);
            }
        } else if (t == T_PHIZ) {
            const cplx<TB>* ps = col0 + PL_S6 * pstride;
            const cplx<TB>* pa = col0 + PL_A * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, ps += step, pa += step) {
                const C s = cv(ld_stream(ps)), av = cv(ld_ordered(pa));
                const TF kzv = kzs * (TF)signed_bin(lane + N2 * m, N);
                v[m] = mk(s.x + nu2 * kzv * av.y, s.y - nu2 * kzv * av.x);
                r[m] = mk(r[m].x - kzv * v[m].y, r[m].y + kzv * v[m].x);
            }
        } else if (t == T_XI) {
            const cplx<TB>* px = col0 + PL_XI * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, px += step) {
                v[m] = cv(ld_stream(px));
                r[m] = r[m] - v[m];
            }
        } else if (t == T_RES) {
            #pragma unroll
            for (int m = 0; m < N1; ++m) v[m] = r[m];
        } else {
            const cplx<TB>* pj = col0 + (t == T_PHIY ? PL_PHIY : PL_PHI) * pstride;
            #pragma unroll
            for (int m = 0; m < N1; ++m, pj += step) v[m] = cv(ld_stream(pj));
        }
        if (!out) continue;
        __syncthreads();                     // exchange buffer free (twiddles ready)
        fft2l<TF, N1, N2, true>(v, lane, xs + c, N2 * CW + 1, CW, stw);
        if (live) {
            C* dst = W + (long long)t * nrz * nxh * pchunk + (long long)kx * pchunk + pl;
            #pragma unroll
            for (int m = 0; m < N1; ++m) {
                const int zr = US ? sm.zrow(lane + N2 * m) : lane + N2 * m;
                if (zr >= 0) dst[(long long)zr * nxh * pchunk] = v[m];
            }
        }
    }
}

// row pass from Wp, four pairs per sequence group: CTA = 4 consecutive pairs x
// N2 lanes x 4 kept z rows (256 threads); a warp holds 4 pairs x 8 lanes of one
// row, so its loads of Wp (4 pairs at 8 kx) and its stores of the terms (4
// pairs x 8 consecutive separations) are whole 32-byte sectors.  The exchange
// regions of the (row, pair) sequences are 4 mod 16 complex values apart, so
// a half-warp (4 pairs x 4 lanes) hits 16 distinct bank pairs.
template <typename TF, typename TO, int N1, int N2, bool US>
__global__ void __launch_bounds__(256, 4)
k_terms_rowpass_p4(const cplx<TF>* __restrict__ W, const int* __restrict__ pair_i, long long pair0,
                   long long npair, long long pchunk, int ny, double inv_count, const double* __restrict__ prof,
                   const cplx<TF>* __restrict__ tw_x, SepMap sm, unsigned tmask, TO* __restrict__ terms,
                   float* __restrict__ spec)
{
    typedef cplx<TF> C;
    constexpr int N = N1 * N2, nxh = N / 2 + 1, NP = 4, NR = 256 / (NP * N2);
    constexpr int REG = N1 * (N2 + 1) + 4;            // exchange region of one sequence (4 mod 16)
    static_assert(REG % 16 == 4 && NR >= 1, "exchange layout");
    extern __shared__ __align__(16) unsigned char sh_raw_rp4[];
    C* stw = (C*)sh_raw_rp4;
    C* xs = stw + N;
    __shared__ TF s_one[NP][NTERM];
    const int c = threadIdx.x % NP, lane = (threadIdx.x / NP) % N2, r = threadIdx.x / (NP * N2);
    const long long pl = (long long)blockIdx.x * NP + c, p = pair0 + pl;
    const bool live = p < npair && pl < pchunk;
    const int nz = sm.nrz, nrx = US ? sm.nrx : N;
    const int zr = blockIdx.y * NR + r;
    const bool zlive = zr < nz;
    load_twiddles(stw, tw_x, N);
    if (threadIdx.x < NP) {
        const long long pp = pair0 + (long long)blockIdx.x * NP + threadIdx.x;
        double one[NTERM] = {0, 0, 0, 0, 0, 0, 0};
        if (pp < npair && (long long)blockIdx.x * NP + threadIdx.x < pchunk)
            onepoint(prof, ny, pair_i[2 * pp], pair_i[2 * pp + 1], one);
        for (int t = 0; t < NTERM; ++t) s_one[threadIdx.x][t] = (TF)one[t];
    }
    const TF ic = (TF)inv_count;
    const long long NN = (long long)nz * nrx;
    const long long tstride = (long long)nz * nxh * pchunk;
    const C* wrow = W + (long long)(zlive ? zr : 0) * nxh * pchunk + pl;
    C* xr = xs + (r * NP + c) * REG;
    for (int jq = 0; jq < 4; ++jq) {
        const int ta = 2 * jq, tb = 2 * jq + 1;
        const bool ha = (tmask >> ta) & 1u, hb = tb < NTERM && ((tmask >> tb) & 1u);
        if (!ha && !hb) continue;                   // uniform over the CTA
        const C* wa = wrow + ta * tstride;
        const C* wb = wrow + (tb < NTERM ? tb : ta) * tstride;
        C v[N1];
        #pragma unroll
        for (int m = 0; m < N1; ++m) {
            const int k = lane + N2 * m;
            C A = mk((TF)0, (TF)0), B = A;           // terms outside tmask: zero, not stale W
            if (live && zlive) {
                const long long off = (long long)(k < nxh ? k : N - k) * pchunk;
                if (ha) A = wa[off];
                if (hb) B = wb[off];
                if (k >= nxh) { A.y = -A.y; B.y = -B.y; }
            }
            if (k == 0 || 2 * k == N) { A.y = 0; B.y = 0; }
            v[m] = mk(A.x - B.y, A.y + B.x);
        }
        __syncthreads();                     // exchange buffer free (and s_one, twiddles ready)
        fft2l<TF, N1, N2, true>(v, lane, xr, N2 + 1, 1, stw);
        if (live && zlive) {
            #pragma unroll
            for (int m = 0; m < N1; ++m) {
                const int x = lane + N2 * m;
                const int xo = US ? sm.xcol(x) : x;
                if (xo < 0) continue;
                const long long e = (long long)zr * nrx + xo;
                #pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = 2 * jq + h;
                    if (q >= NTERM) break;
                    if (!(h ? hb : ha)) continue;
                    const TF sp = (h ? v[m].y : v[m].x) * ic;
                    if (spec == nullptr || (q != T_PHIY && q != T_PHI))
                        st_stream(terms + ((long long)q * npair + p) * NN + e, (TO)(sp + s_one[c][q]));
                    if (spec != nullptr) {
                        const int si = (q == T_A) ? 0 : (q == T_PHIY) ? 1 : (q == T_PHI) ? 2 : -1;
                        if (si >= 0) st_stream(spec + ((long long)si * npair + p) * NN + e, (float)sp);
                    }
                }
            }
        }
    }
}

// the plane-mode column pass of one pair chunk (FP32 transforms only)
template <typename TF, typename TB>
static void colpass_planes_launch(const TermArgs& a, long long p0, long long np, cplx<TF>* W, cudaStream_t sc,
                                  bool us)
{
    if constexpr (sizeof(TF) == 4) {
        typedef cplx<TF> C;
        const int nxh = a.nx / 2 + 1;
        PlaneCols pc{a.planes, a.npp, a.Kc, a.pair_i, a.prof, a.ny, a.Lx, a.Lz, a.nu};
        if (a.nz == 256 && a.nx == 256) {
            // pair-contiguous W (k_terms_rowpass_p4 reads it)
            const dim3 g((unsigned)((np + 15) / 16), nxh);
            const size_t sh = (256 + 16 * (16 * 16 + 1)) * sizeof(C);
            if (us)
                k_terms_colpass_pt<TF, TB, 16, 16, true><<<g, 256, sh, sc>>>(pc, p0, a.npair, a.pair_chunk, a.nx,
                                                                            (const C*)a.tw_z, a.sep, a.tmask, W);
            else
                k_terms_colpass_pt<TF, TB, 16, 16, false><<<g, 256, sh, sc>>>(pc, p0, a.npair, a.pair_chunk, a.nx,
                                                                             (const C*)a.tw_z, a.sep, a.tmask, W);
        } else if (a.nz == 256) {
            const dim3 g((unsigned)((np + 3) / 4), (nxh + 3) / 4);
            const size_t sh = (256 + 16 * (16 * 16 + 1)) * sizeof(C);
            if (us)
                k_terms_colpass_planes_r<TF, TB, 16, 16, true><<<g, 256, sh, sc>>>(
                    pc, p0, a.npair, a.nx, (const C*)a.tw_z, a.sep, a.tmask, W);
            else
                k_terms_colpass_planes_r<TF, TB, 16, 16, false><<<g, 256, sh, sc>>>(
                    pc, p0, a.npair, a.nx, (const C*)a.tw_z, a.sep, a.tmask, W);
        } else {
            const int kxc = planes_kxc(a.nz, sizeof(C));
            const dim3 g((unsigned)((np + 3) / 4), (nxh + kxc - 1) / kxc);
            k_terms_colpass_planes<TF, TB><<<g, 256, (size_t)(1 + 3 * 4 * kxc) * a.nz * sizeof(C), sc>>>(
                pc, p0, a.npair, a.nz, a.nx, kxc, (const C*)a.tw_z, a.sep, a.tmask, W);
        }
    }
}

// the row pass from the pair-contiguous W of k_terms_colpass_pt
template <typename TF, typename TO>
static void rowpass_pt_launch(const TermArgs& a, long long p0, long long np, const cplx<TF>* W, cudaStream_t sr,
                              bool us)
{
    if constexpr (sizeof(TF) == 4) {
        typedef cplx<TF> C;
        // 4 pairs x 4 rows per CTA
        const dim3 g((unsigned)((np + 3) / 4), (unsigned)((a.sep.nrz + 3) / 4));
        const size_t sh = (256 + 16 * (16 * 17 + 4)) * sizeof(C);
        if (us)
            k_terms_rowpass_p4<TF, TO, 16, 16, true><<<g, 256, sh, sr>>>(
                W, a.pair_i, p0, a.npair, a.pair_chunk, a.ny, a.inv_count, a.prof, (const C*)a.tw_x, a.sep, a.tmask,
                (TO*)a.terms, a.spec);
        else
            k_terms_rowpass_p4<TF, TO, 16, 16, false><<<g, 256, sh, sr>>>(
                W, a.pair_i, p0, a.npair, a.pair_chunk, a.ny, a.inv_count, a.prof, (const C*)a.tw_x, a.sep, a.tmask,
                (TO*)a.terms, a.spec);
    }
}

template <typename TF, typename TB, typename TO>
int terms_launch_t(const TermArgs& a)
{
    typedef cplx<TF> C;
    const int nxh = a.nx / 2 + 1;
    const bool us = a.sep.zpos != nullptr || a.sep.xpos != nullptr;      // undersampled output
    // With a second stream and a second scratch buffer, the column pass of
    // chunk c + 1 runs on a.st while the row pass of chunk c runs on a.st2:
    // the GPU stays full with chunks small enough for W to stay in L2.
    const bool two = a.st2 != nullptr && a.W2 != nullptr;
    cudaEvent_t ev_col[2] = {nullptr, nullptr}, ev_row[2] = {nullptr, nullptr};
    if (two) {
        if (a.ev) {
            ev_col[0] = a.ev[0]; ev_col[1] = a.ev[1]; ev_row[0] = a.ev[2]; ev_row[1] = a.ev[3];
        } else {
            for (int i = 0; i < 2; ++i) {
                cudaEventCreateWithFlags(&ev_col[i], cudaEventDisableTiming);
                cudaEventCreateWithFlags(&ev_row[i], cudaEventDisableTiming);
            }
        }
    }
    int launches = 0;
    const unsigned ntm = (unsigned)__builtin_popcount(a.tmask);     // column passes: the terms of tmask
    long long c = 0;
    for (long long p0 = 0; p0 < a.npair; p0 += a.pair_chunk, ++c) {
        const long long np = a.pair_chunk < a.npair - p0 ? a.pair_chunk : a.npair - p0;
        const int buf = two ? (int)(c & 1) : 0;
        C* W = (C*)(buf ? a.W2 : a.W);
        cudaStream_t sc = a.st, sr = two ? a.st2 : a.st;
        if (two && c >= 2) cudaStreamWaitEvent(sc, ev_row[buf], 0);     // W buffer free again
        if (a.planes) {
            colpass_planes_launch<TF, TB>(a, p0, np, W, sc, us);        } else if (a.nz == 256) {
            constexpr int CWR = 16;
            const dim3 g((nxh + CWR - 1) / CWR, ntm, (unsigned)np);
            const size_t sh = (256 + 16 * (16 * CWR + 1)) * sizeof(C);
            if (us)
                k_terms_colpass_r<TF, TB, 16, 16, true><<<g, CWR * 16, sh, sc>>>(
                    (const cplx<TB>*)a.comb, p0, nxh, CWR, (const C*)a.tw_z, a.sep, a.tmask, W);
            else
                k_terms_colpass_r<TF, TB, 16, 16, false><<<g, CWR * 16, sh, sc>>>(
                    (const cplx<TB>*)a.comb, p0, nxh, CWR, (const C*)a.tw_z, a.sep, a.tmask, W);
        } else {
            k_terms_colpass<TF, TB><<<dim3((nxh + a.cw - 1) / a.cw, ntm, (unsigned)np), 256,
                                      (1 + 2 * a.cw) * a.nz * sizeof(C), sc>>>(
                (const cplx<TB>*)a.comb, p0, a.nz, a.nx, a.cw, (const C*)a.tw_z, a.sep, a.tmask, W);
        }
        if (two) {
            cudaEventRecord(ev_col[buf], sc);
            cudaStreamWaitEvent(sr, ev_col[buf], 0);
        }
        if (sizeof(TF) == 4 && a.planes && a.nz == 256 && a.nx == 256) {
            rowpass_pt_launch<TF, TO>(a, p0, np, W, sr, us);
        } else if (a.nx == 256) {
            constexpr int RZR = 4;
            const dim3 g((a.sep.nrz + RZR - 1) / RZR, (unsigned)np);
            const size_t sh = (256 + RZR * 16 * 17) * sizeof(C);
            if (us)
                k_terms_rowpass_r<TF, TO, 16, 16, true><<<g, RZR * 16, sh, sr>>>(
                    W, a.pair_i, p0, a.npair, a.ny, RZR, a.inv_count, a.prof, (const C*)a.tw_x, a.sep,
                    a.tmask, (TO*)a.terms, a.spec);
            else
                k_terms_rowpass_r<TF, TO, 16, 16, false><<<g, RZR * 16, sh, sr>>>(
                    W, a.pair_i, p0, a.npair, a.ny, RZR, a.inv_count, a.prof, (const C*)a.tw_x, a.sep,
                    a.tmask, (TO*)a.terms, a.spec);
        } else {
            k_terms_rowpass<TF, TO><<<dim3((a.sep.nrz + a.rz - 1) / a.rz, (unsigned)np), 256,
                                      (1 + 8 * a.rz) * a.nx * sizeof(C), sr>>>(
                W, a.pair_i, p0, a.npair, a.ny, a.nx, a.rz, a.inv_count, a.prof, (const C*)a.tw_x,
                a.sep, a.tmask, (TO*)a.terms, a.spec);
        }
        if (two) cudaEventRecord(ev_row[buf], sr);
        launches += 2;
        if (a.after_chunk) a.after_chunk(a.ctx, p0, np, sr);
    }
    if (two) {
        // join: the main stream waits for the last row passes
        cudaStreamWaitEvent(a.st, ev_row[0], 0);
        if (c > 1) cudaStreamWaitEvent(a.st, ev_row[1], 0);
        if (!a.ev)
            for (int i = 0; i < 2; ++i) {
                cudaEventDestroy(ev_col[i]);
                cudaEventDestroy(ev_row[i]);
            }
    }
    return launches;
}

int terms_launch(const TermArgs& a)
{
    if (!a.fp32) return terms_launch_t<double, double, double>(a);
    if (a.planes ? a.planes64 : a.comb64) return terms_launch_t<float, double, float>(a);
    return terms_launch_t<float, float, float>(a);
}

cudaError_t terms_set_attrs(int lim)
{
    const void* ks[] = {(const void*)k_terms_colpass<double, double>, (const void*)k_terms_rowpass<double, double>,
                        (const void*)k_terms_colpass<float, float>, (const void*)k_terms_colpass<float, double>,
                        (const void*)k_terms_rowpass<float, float>,
                        (const void*)k_terms_colpass_r<double, double, 16, 16, false>,
                        (const void*)k_terms_colpass_r<float, float, 16, 16, false>,
                        (const void*)k_terms_colpass_r<float, double, 16, 16, false>,
                        (const void*)k_terms_rowpass_r<double, double, 16, 16, false>,
                        (const void*)k_terms_rowpass_r<float, float, 16, 16, false>,
                        (const void*)k_terms_colpass_r<double, double, 16, 16, true>,
                        (const void*)k_terms_colpass_r<float, float, 16, 16, true>,
                        (const void*)k_terms_colpass_r<float, double, 16, 16, true>,
                        (const void*)k_terms_rowpass_r<double, double, 16, 16, true>,
                        (const void*)k_terms_rowpass_r<float, float, 16, 16, true>,
                        (const void*)k_terms_colpass_planes_r<float, float, 16, 16, false>,
                        (const void*)k_terms_colpass_planes_r<float, double, 16, 16, false>,
                        (const void*)k_terms_colpass_planes_r<float, float, 16, 16, true>,
                        (const void*)k_terms_colpass_planes_r<float, double, 16, 16, true>,
                        (const void*)k_terms_colpass_planes<float, float>,
                        (const void*)k_terms_colpass_planes<float, double>,
                        (const void*)k_terms_colpass_pt<float, float, 16, 16, false>,
                        (const void*)k_terms_colpass_pt<float, double, 16, 16, false>,
                        (const void*)k_terms_colpass_pt<float, float, 16, 16, true>,
                        (const void*)k_terms_colpass_pt<float, double, 16, 16, true>,
                        (const void*)k_terms_rowpass_p4<float, float, 16, 16, false>,
                        (const void*)k_terms_rowpass_p4<float, float, 16, 16, true>};
    cudaError_t e = cudaSuccess;
    for (const void* k : ks) {
        cudaFuncAttributes fa;
        cudaError_t r = cudaFuncGetAttributes(&fa, k);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - (int)fa.sharedSizeBytes);
        if (r != cudaSuccess) e = r;
    }
    return e;
}

// ----------------------------------------------- Step 3 FD stencils
// value of a field at the ordered pair (a, b) and separation index
// (mz, mx), taken from the stored triangle a <= b, or by r-inversion
// (Sec. 3.3) with parity sg
// v or -v by flipping the sign bit with an integer operation (no FP64 work)
__device__ __forceinline__ double flip_sign(double v, bool neg)
{
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}

template <bool WEDGE, bool US, typename T>
__device__ __forceinline__ T tri_value(const T* __restrict__ f, int a, int b, int ny, const SepMap& sm,
                                       int zr, int xr, int rho, int sigma)
{
    const long long N = (long long)sm.nrz * sm.nrx;
    int sg;                             // integer parities: no FP64 work per gather
    bool flip;
    const long long q = stored_pair(a, b, ny, WEDGE, rho, sigma, sg, flip);
    T v;
    if (!flip) v = f[q * N + (long long)zr * sm.nrx + xr];
    else if (US) v = f[q * N + (long long)sm.negz[zr] * sm.nrx + sm.negx[xr]];
    else v = f[q * N + (long long)((sm.nz - zr) % sm.nz) * sm.nx + (sm.nx - xr) % sm.nx];
    return flip_sign(v, sg < 0);
}

// plain path, pass 1: Phi_y -= 2 nu dA/dr_y, phi -= (nu/2) dA/dY, with
// dA/dr_y = (d_Y2 - d_Y1) A / 2, dA/dY = (d_Y1 + d_Y2) A (Eq. 10-11); A even
// under r-inversion and under the combined inversion.  grid (npair,
// separation chunks): consecutive CTAs take the same separation chunk of
// consecutive pairs, so neighbour rows stay in L2.
template <bool WEDGE, bool US>
__global__ void k_stencil_A(double* __restrict__ terms, long long npair, const int* __restrict__ pair_i,
                            int ny, SepMap sm, double nu, const double* __restrict__ fdw,
                            const int* __restrict__ fdl0)
{
    const long long N = (long long)sm.nrz * sm.nrx;
    const long long p = blockIdx.x;
    const long long e = (long long)blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int mz = (int)(e / sm.nrx), mx = (int)(e - (long long)mz * sm.nrx);
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    const double* A = terms + (long long)T_A * npair * N;
    double d1 = 0.0, d2 = 0.0;
    const int a1 = fdl0[i1], a2 = fdl0[i2];
    #pragma unroll
    for (int l = 0; l < 5; ++l) {
        d1 += fdw[5 * i1 + l] * tri_value<WEDGE, US>(A, a1 + l, i2, ny, sm, mz, mx, 1, 1);
        d2 += fdw[5 * i2 + l] * tri_value<WEDGE, US>(A, i1, a2 + l, ny, sm, mz, mx, 1, 1);
    }
    terms[((long long)T_PHIY * npair + p) * N + e] += -2.0 * nu * 0.5 * (d2 - d1);
    terms[((long long)T_PHI * npair + p) * N + e] += -0.5 * nu * (d1 + d2);
}

// plain path, pass 2: res += dPhi_y/dr_y + dphi/dY by the same stencil;
// Phi_y odd and phi even under r-inversion, Phi_y even and phi odd under the
// combined inversion.
template <bool WEDGE, bool US>
__global__ void k_stencil_res(double* __restrict__ terms, long long npair, const int* __restrict__ pair_i,
                              int ny, SepMap sm, const double* __restrict__ fdw,
                              const int* __restrict__ fdl0)
{
    const long long N = (long long)sm.nrz * sm.nrx;
    const long long p = blockIdx.x;
    const long long e = (long long)blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int mz = (int)(e / sm.nrx), mx = (int)(e - (long long)mz * sm.nrx);
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    const double* Py = terms + (long long)T_PHIY * npair * N;
    const double* Ph = terms + (long long)T_PHI * npair * N;
    double y1 = 0.0, y2 = 0.0, h1 = 0.0, h2 = 0.0;
    const int a1 = fdl0[i1], a2 = fdl0[i2];
    #pragma unroll
    for (int l = 0; l < 5; ++l) {
        double w1 = fdw[5 * i1 + l], w2 = fdw[5 * i2 + l];
        y1 += w1 * tri_value<WEDGE, US>(Py, a1 + l, i2, ny, sm, mz, mx, -1, 1);
        y2 += w2 * tri_value<WEDGE, US>(Py, i1, a2 + l, ny, sm, mz, mx, -1, 1);
        h1 += w1 * tri_value<WEDGE, US>(Ph, a1 + l, i2, ny, sm, mz, mx, 1, -1);
        h2 += w2 * tri_value<WEDGE, US>(Ph, i1, a2 + l, ny, sm, mz, mx, 1, -1);
    }
    terms[((long long)T_RES * npair + p) * N + e] += 0.5 * (y2 - y1) + (h1 + h2);
}

// ------------------------------------- split path: FP32 stencils
// One-point part of A, a function of the ordered pair only
__device__ __forceinline__ double op_A(const double* pr, int ny, int a, int b)
{
    return pr[PR_Q * ny + a] + pr[PR_Q * ny + b];
}

// final one-point parts of Phi_y and phi at the ordered pair (a, b), their FD
// parts included (FP64)
__device__ __forceinline__ void op_final(const double* pr, int ny, double nu, const double* fdw, const int* fdl0,
                                         int a, int b, double& py, double& ph)
{
    const int la = fdl0[a], lb = fdl0[b];
    double d1 = 0.0, d2 = 0.0;
    for (int l = 0; l < 5; ++l) {
        d1 += fdw[5 * a + l] * op_A(pr, ny, la + l, b);
        d2 += fdw[5 * b + l] * op_A(pr, ny, a, lb + l);
    }
    const double qv_a = pr[PR_QV * ny + a], qv_b = pr[PR_QV * ny + b];
    const double pv_a = pr[PR_PV * ny + a], pv_b = pr[PR_PV * ny + b];
    py = (qv_b - qv_a) - nu * (d2 - d1);
    ph = 0.5 * (qv_a + qv_b) + 2.0 * (pv_a + pv_b) - 0.5 * nu * (d1 + d2);
}

// Per-pair scalars of the split stencils, computed once in FP64:
//   sc[p] = { w1[0..5), w2[0..5) (FP32 copies of the FD weights of rows i1, i2),
//             -nu (d_Y2 - d_Y1) A1, -(nu/2) (d_Y1 + d_Y2) A1,
//             (d_Y2 - d_Y1) Phi_y1 / 2 + (d_Y1 + d_Y2) phi1,
//             the one-point parts of Phi_y and phi that the row pass adds
//             to the other terms }
// with A1, Phi_y1, phi1 the one-point parts (FD parts included).
constexpr int NSC = 15;
__global__ void k_stencil_pairs(const int* __restrict__ pair_i, long long npair, int ny, double nu,
                                const double* __restrict__ fdw, const int* __restrict__ fdl0,
                                const double* __restrict__ prof, float* __restrict__ sc)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npair) return;
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    const int a1 = fdl0[i1], a2 = fdl0[i2];
    double d1 = 0.0, d2 = 0.0, y1 = 0.0, y2 = 0.0, h1 = 0.0, h2 = 0.0;
    for (int l = 0; l < 5; ++l) {
        const double w1 = fdw[5 * i1 + l], w2 = fdw[5 * i2 + l];
        d1 += w1 * op_A(prof, ny, a1 + l, i2);
        d2 += w2 * op_A(prof, ny, i1, a2 + l);
        double py, ph;
        op_final(prof, ny, nu, fdw, fdl0, a1 + l, i2, py, ph);
        y1 += w1 * py;
        h1 += w1 * ph;
        op_final(prof, ny, nu, fdw, fdl0, i1, a2 + l, py, ph);
        y2 += w2 * py;
        h2 += w2 * ph;
        sc[p * NSC + l] = (float)w1;
        sc[p * NSC + 5 + l] = (float)w2;
    }
    sc[p * NSC + 10] = (float)(-nu * (d2 - d1));
    sc[p * NSC + 11] = (float)(-0.5 * nu * (d1 + d2));
    sc[p * NSC + 12] = (float)(0.5 * (y2 - y1) + (h1 + h2));
    double one[NTERM];
    onepoint(prof, ny, i1, i2, one);
    sc[p * NSC + 13] = (float)one[T_PHIY];
    sc[p * NSC + 14] = (float)one[T_PHI];
}

constexpr int SPT = 4;   // separations per thread in the split stencils

// the stencil's 10 neighbours of pair (i1, i2): rows (a1 + l, i2) and columns
// (i1, a2 + l); a neighbour outside the stored pairs is read from the stored
// pair that the inversions map it to (stored_pair: sign, inverted
// separation).  Resolved once per CTA so the per-separation gathers are
// branch-free.
struct Nb { const float* base[10]; float sg[10]; int mir[10]; };

template <bool WEDGE>
__device__ __forceinline__ void make_nb(Nb& nb, const float* f, float rho, float sigma, int i1, int i2, int a1,
                                        int a2, int ny, long long N)
{
    #pragma unroll
    for (int l = 0; l < 10; ++l) {
        const int a = l < 5 ? a1 + l : i1, b = l < 5 ? i2 : a2 + (l - 5);
        float sg;
        bool flip;
        nb.base[l] = f + stored_pair(a, b, ny, WEDGE, rho, sigma, sg, flip) * N;
        nb.sg[l] = sg;
        nb.mir[l] = flip;
    }
}

// pass 1, FP32: with S = spectral part of A (spec[0]),
//   Phi_y = spec[1] + one-point + -nu (d_Y2 - d_Y1)(S + A1),
//   phi = spec[2] + one-point + -(nu/2) (d_Y1 + d_Y2)(S + A1)
// (written for the terms in tmask); spec[1], spec[2] (spectral parts of
// Phi_y, phi) receive the FD parts of S.
// grid (npair, separation chunks of 256 SPT).
template <bool WEDGE, bool US>
__global__ void k_stencil_A32(float* __restrict__ terms, float* __restrict__ spec, long long npair,
                              const int* __restrict__ pair_i, int ny, SepMap sm, double nu,
                              const int* __restrict__ fdl0, const float* __restrict__ sc, unsigned tmask)
{
    const long long N = (long long)sm.nrz * sm.nrx;
    const long long p = blockIdx.x;
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    float w[10];
    #pragma unroll
    for (int l = 0; l < 10; ++l) w[l] = sc[p * NSC + l];
    const float oy = sc[p * NSC + 10], oh = sc[p * NSC + 11];
    const float nuf = (float)nu;
    Nb nb;
    make_nb<WEDGE>(nb, spec, 1.f, 1.f, i1, i2, fdl0[i1], fdl0[i2], ny, N);
    #pragma unroll
    for (int u = 0; u < SPT; ++u) {
        const long long e = ((long long)blockIdx.y * SPT + u) * blockDim.x + threadIdx.x;
        if (e >= N) return;
        const int mz = (int)(e / sm.nrx), mx = (int)(e - (long long)mz * sm.nrx);
        const long long en = US ? (long long)sm.negz[mz] * sm.nrx + sm.negx[mx]
                                : (long long)((sm.nz - mz) % sm.nz) * sm.nx + (sm.nx - mx) % sm.nx;
        float d1 = 0.f, d2 = 0.f;
        #pragma unroll
        for (int l = 0; l < 5; ++l) {
            d1 = fmaf(w[l] * nb.sg[l], nb.base[l][nb.mir[l] ? en : e], d1);
            d2 = fmaf(w[5 + l] * nb.sg[5 + l], nb.base[5 + l][nb.mir[5 + l] ? en : e], d2);
        }
        // products rounded on their own (no contraction into the sums below),
        // as in k_stencil_A32q, so the two kernels give bit-equal values
        const float fy = __fmul_rn(-nuf, d2 - d1), fp = __fmul_rn(-0.5f * nuf, d1 + d2);
        float* s1 = spec + ((long long)1 * npair + p) * N + e;
        float* s2 = spec + ((long long)2 * npair + p) * N + e;
        const float v1 = *s1, v2 = *s2;
        if ((tmask >> T_PHIY) & 1u) terms[((long long)T_PHIY * npair + p) * N + e] = (v1 + sc[p * NSC + 13]) + (fy + oy);
        if ((tmask >> T_PHI) & 1u) terms[((long long)T_PHI * npair + p) * N + e] = (v2 + sc[p * NSC + 14]) + (fp + oh);
        *s1 = v1 + fy;
        *s2 = v2 + fp;
    }
}

// pass 2, FP32: res += (d_Y2 - d_Y1) Phi_y / 2 + (d_Y1 + d_Y2) phi, the
// spectral parts (spec[1] odd, spec[2] even) in FP32 plus the per-pair
// one-point scalar.
template <bool WEDGE, bool US>
__global__ void k_stencil_res32(float* __restrict__ terms, const float* __restrict__ spec, long long npair,
                                const int* __restrict__ pair_i, int ny, SepMap sm,
                                const int* __restrict__ fdl0, const float* __restrict__ sc)
{
    const long long N = (long long)sm.nrz * sm.nrx;
    const long long p = blockIdx.x;
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    float w[10];
    #pragma unroll
    for (int l = 0; l < 10; ++l) w[l] = sc[p * NSC + l];
    const float o = sc[p * NSC + 12];
    Nb ny_, nh_;
    make_nb<WEDGE>(ny_, spec + (long long)1 * npair * N, -1.f, 1.f, i1, i2, fdl0[i1], fdl0[i2], ny, N);
    make_nb<WEDGE>(nh_, spec + (long long)2 * npair * N, 1.f, -1.f, i1, i2, fdl0[i1], fdl0[i2], ny, N);
    #pragma unroll
    for (int u = 0; u < SPT; ++u) {
        const long long e = ((long long)blockIdx.y * SPT + u) * blockDim.x + threadIdx.x;
        if (e >= N) return;
        const int mz = (int)(e / sm.nrx), mx = (int)(e - (long long)mz * sm.nrx);
        const long long en = US ? (long long)sm.negz[mz] * sm.nrx + sm.negx[mx]
                                : (long long)((sm.nz - mz) % sm.nz) * sm.nx + (sm.nx - mx) % sm.nx;
        float y1 = 0.f, y2 = 0.f, h1 = 0.f, h2 = 0.f;
        #pragma unroll
        for (int l = 0; l < 5; ++l) {
            y1 = fmaf(w[l] * ny_.sg[l], ny_.base[l][ny_.mir[l] ? en : e], y1);
            y2 = fmaf(w[5 + l] * ny_.sg[5 + l], ny_.base[5 + l][ny_.mir[5 + l] ? en : e], y2);
            h1 = fmaf(w[l] * nh_.sg[l], nh_.base[l][nh_.mir[l] ? en : e], h1);
            h2 = fmaf(w[5 + l] * nh_.sg[5 + l], nh_.base[5 + l][nh_.mir[5 + l] ? en : e], h2);
        }
        terms[((long long)T_RES * npair + p) * N + e] += __fadd_rn(fmaf(0.5f, y2 - y1, h1 + h2), o);
    }
}

// Full separation grid (nx a multiple of 4): the same two passes with each
// thread on four consecutive r_x of one r_z row, so a stored neighbour is
// one 16-byte load and the row / column indices take no division per value;
// an r-inverted neighbour reads its four values at -r one by one.
__device__ __forceinline__ float4 nb_quad(const float* b, bool mir, long long e0, long long enb, int nx, int mx0)
{
    if (!mir) return *(const float4*)(b + e0);
    return make_float4(b[enb + (mx0 == 0 ? 0 : nx - mx0)], b[enb + nx - mx0 - 1], b[enb + nx - mx0 - 2],
                       b[enb + nx - mx0 - 3]);
}
__device__ __forceinline__ void fma4(float4& a, float c, float4 v)
{
    a.x = fmaf(c, v.x, a.x); a.y = fmaf(c, v.y, a.y); a.z = fmaf(c, v.z, a.z); a.w = fmaf(c, v.w, a.w);
}
__device__ __forceinline__ void add4(float* dst, float4 v)
{
    float4 o = *(float4*)dst;
    o.x += v.x; o.y += v.y; o.z += v.z; o.w += v.w;
    *(float4*)dst = o;
}

template <bool WEDGE>
__global__ void __launch_bounds__(256)
k_stencil_A32q(float* __restrict__ terms, float* __restrict__ spec, long long npair, const int* __restrict__ pair_i,
               int ny, int nz, int nx, double nu, const int* __restrict__ fdl0, const float* __restrict__ sc,
               unsigned tmask)
{
    const long long N = (long long)nz * nx;
    const long long p = blockIdx.x;
    const long long e0 = ((long long)blockIdx.y * blockDim.x + threadIdx.x) * 4;
    if (e0 >= N) return;
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    Nb nb;
    make_nb<WEDGE>(nb, spec, 1.f, 1.f, i1, i2, fdl0[i1], fdl0[i2], ny, N);
    const int mz = (int)(e0 / nx), mx0 = (int)(e0 - (long long)mz * nx);
    const long long enb = (long long)((nz - mz) % nz) * nx;
    float4 d1 = make_float4(0.f, 0.f, 0.f, 0.f), d2 = d1;
    #pragma unroll
    for (int l = 0; l < 5; ++l) {
        fma4(d1, sc[p * NSC + l] * nb.sg[l], nb_quad(nb.base[l], nb.mir[l], e0, enb, nx, mx0));
        fma4(d2, sc[p * NSC + 5 + l] * nb.sg[5 + l], nb_quad(nb.base[5 + l], nb.mir[5 + l], e0, enb, nx, mx0));
    }
    const float oy = sc[p * NSC + 10], oh = sc[p * NSC + 11];
    const float a = -(float)nu, b = -0.5f * (float)nu;
    const float4 fy = make_float4(__fmul_rn(a, d2.x - d1.x), __fmul_rn(a, d2.y - d1.y), __fmul_rn(a, d2.z - d1.z),
                                  __fmul_rn(a, d2.w - d1.w));
    const float4 fp = make_float4(__fmul_rn(b, d1.x + d2.x), __fmul_rn(b, d1.y + d2.y), __fmul_rn(b, d1.z + d2.z),
                                  __fmul_rn(b, d1.w + d2.w));
    float4* s1 = (float4*)(spec + ((long long)1 * npair + p) * N + e0);
    float4* s2 = (float4*)(spec + ((long long)2 * npair + p) * N + e0);
    const float4 v1 = *s1, v2 = *s2;
    const float ty = sc[p * NSC + 13], th = sc[p * NSC + 14];
    if ((tmask >> T_PHIY) & 1u)
        *(float4*)(terms + ((long long)T_PHIY * npair + p) * N + e0) =
            make_float4((v1.x + ty) + (fy.x + oy), (v1.y + ty) + (fy.y + oy), (v1.z + ty) + (fy.z + oy),
                        (v1.w + ty) + (fy.w + oy));
    if ((tmask >> T_PHI) & 1u)
        *(float4*)(terms + ((long long)T_PHI * npair + p) * N + e0) =
            make_float4((v2.x + th) + (fp.x + oh), (v2.y + th) + (fp.y + oh), (v2.z + th) + (fp.z + oh),
                        (v2.w + th) + (fp.w + oh));
    *s1 = make_float4(v1.x + fy.x, v1.y + fy.y, v1.z + fy.z, v1.w + fy.w);
    *s2 = make_float4(v2.x + fp.x, v2.y + fp.y, v2.z + fp.z, v2.w + fp.w);
}

template <bool WEDGE>
__global__ void __launch_bounds__(256)
k_stencil_res32q(float* __restrict__ terms, const float* __restrict__ spec, long long npair,
                 const int* __restrict__ pair_i, int ny, int nz, int nx, const int* __restrict__ fdl0,
                 const float* __restrict__ sc)
{
    // the pair's 20 neighbour rows (base, weight x sign, inverted?) once per CTA
    __shared__ const float* s_base[20];
    __shared__ float s_c[20];
    __shared__ int s_mir[20];
    const long long N = (long long)nz * nx;
    const long long p = blockIdx.x;
    if (threadIdx.x < 20) {
        const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
        const int h = threadIdx.x / 10, l = threadIdx.x % 10;       // h 0: Phi_y, 1: phi
        const int a = l < 5 ? fdl0[i1] + l : i1, b = l < 5 ? i2 : fdl0[i2] + (l - 5);
        float sg;
        bool flip;
        const long long q = stored_pair(a, b, ny, WEDGE, h ? 1.f : -1.f, h ? -1.f : 1.f, sg, flip);
        s_base[threadIdx.x] = spec + ((long long)(1 + h) * npair + q) * N;
        s_c[threadIdx.x] = sc[p * NSC + l] * sg;
        s_mir[threadIdx.x] = flip;
    }
    __syncthreads();
    const float o = sc[p * NSC + 12];
    // 0.5 (d_Y2 - d_Y1) Phi_y + (d_Y1 + d_Y2) phi, in the order of k_stencil_res32
    // (the a-posteriori separation selection, which runs that kernel, keeps
    // bit-equal values); two quads per thread
    #pragma unroll
    for (int u = 0; u < 2; ++u) {
        const long long e0 = (((long long)blockIdx.y * 2 + u) * blockDim.x + threadIdx.x) * 4;
        if (e0 < N) {
            const int mz = (int)(e0 / nx), mx0 = (int)(e0 - (long long)mz * nx);
            const long long enb = (long long)((nz - mz) % nz) * nx;
            float4 y1 = make_float4(0.f, 0.f, 0.f, 0.f), y2 = y1, h1 = y1, h2 = y1;
            #pragma unroll
            for (int l = 0; l < 5; ++l) {
                fma4(y1, s_c[l], nb_quad(s_base[l], s_mir[l], e0, enb, nx, mx0));
                fma4(y2, s_c[5 + l], nb_quad(s_base[5 + l], s_mir[5 + l], e0, enb, nx, mx0));
                fma4(h1, s_c[10 + l], nb_quad(s_base[10 + l], s_mir[10 + l], e0, enb, nx, mx0));
                fma4(h2, s_c[15 + l], nb_quad(s_base[15 + l], s_mir[15 + l], e0, enb, nx, mx0));
            }
            auto r = [&](float a1, float a2, float b1, float b2) { return __fadd_rn(fmaf(0.5f, a2 - a1, b1 + b2), o); };
            add4(terms + ((long long)T_RES * npair + p) * N + e0,
                 make_float4(r(y1.x, y2.x, h1.x, h2.x), r(y1.y, y2.y, h1.y, h2.y), r(y1.z, y2.z, h1.z, h2.z),
                             r(y1.w, y2.w, h1.w, h2.w)));
        }
    }
}

template <bool WEDGE, bool US>
static int stencil_launch_t(bool fp32, void* terms, float* spec, long long npair, const int* pair_i, int ny,
                            const SepMap& sm, double nu, const double* fdw, const int* fdl0, const double* prof,
                            unsigned tmask, cudaStream_t st)
{
    // Phi_y and phi take the FD parts of A; the residual those of Phi_y and phi
    const bool pass1 = (tmask & ((1u << T_PHIY) | (1u << T_PHI))) != 0, pass2 = ((tmask >> T_RES) & 1u) != 0;
    if (!pass1) return 0;
    const long long N = (long long)sm.nrz * sm.nrx;
    dim3 gs((unsigned)npair, (unsigned)((N + 255) / 256));
    if (!fp32) {
        k_stencil_A<WEDGE, US><<<gs, 256, 0, st>>>((double*)terms, npair, pair_i, ny, sm, nu, fdw, fdl0);
        if (!pass2) return 1;
        k_stencil_res<WEDGE, US><<<gs, 256, 0, st>>>((double*)terms, npair, pair_i, ny, sm, fdw, fdl0);
        return 2;
    }
    float* sc = spec + (size_t)3 * npair * N;      // per-pair scalars after the three spectral parts
    k_stencil_pairs<<<(unsigned)((npair + 127) / 128), 128, 0, st>>>(pair_i, npair, ny, nu, fdw, fdl0, prof, sc);
    if (!US && sm.nx % 4 == 0 && ((uintptr_t)terms & 15u) == 0) {
        // one quad per thread in pass 1, two in pass 2 (its 20 neighbour rows
        // resolved once per CTA)
        dim3 g1((unsigned)npair, (unsigned)((N / 4 + 255) / 256)), g2((unsigned)npair, (unsigned)((N / 4 + 511) / 512));
        k_stencil_A32q<WEDGE><<<g1, 256, 0, st>>>((float*)terms, spec, npair, pair_i, ny, sm.nz, sm.nx, nu, fdl0, sc,
                                                  tmask);
        if (!pass2) return 2;
        k_stencil_res32q<WEDGE><<<g2, 256, 0, st>>>((float*)terms, spec, npair, pair_i, ny, sm.nz, sm.nx, fdl0, sc);
        return 3;
    }
    dim3 g32((unsigned)npair, (unsigned)((N + 256 * SPT - 1) / (256 * SPT)));
    k_stencil_A32<WEDGE, US><<<g32, 256, 0, st>>>((float*)terms, spec, npair, pair_i, ny, sm, nu, fdl0, sc, tmask);
    if (!pass2) return 2;
    k_stencil_res32<WEDGE, US><<<g32, 256, 0, st>>>((float*)terms, spec, npair, pair_i, ny, sm, fdl0, sc);
    return 3;
}

int stencil_launch(bool fp32, int wedge, void* terms, float* spec, long long npair, const int* pair_i, int ny,
                   const SepMap& sm, double nu, const double* fdw, const int* fdl0, const double* prof,
                   unsigned tmask, cudaStream_t st)
{
    const bool us = sm.negz != nullptr;
    if (wedge)
        return us ? stencil_launch_t<true, true>(fp32, terms, spec, npair, pair_i, ny, sm, nu, fdw, fdl0, prof, tmask, st)
                  : stencil_launch_t<true, false>(fp32, terms, spec, npair, pair_i, ny, sm, nu, fdw, fdl0, prof, tmask, st);
    return us ? stencil_launch_t<false, true>(fp32, terms, spec, npair, pair_i, ny, sm, nu, fdw, fdl0, prof, tmask, st)
              : stencil_launch_t<false, false>(fp32, terms, spec, npair, pair_i, ny, sm, nu, fdw, fdl0, prof, tmask, st);
}

// ----------------------------------------------- Step-1 mean, on device
// mean = mean_sum / mean_count; with mirror sampling the mean of the
// snapshots and their images (U, W, P even about the centreline, V odd), and
// mean_sum rewritten to match.  One block (both phases need every value).
__global__ void k_freeze_mean(double* __restrict__ mean_sum, double mean_count, int mirror, int ny,
                              double* __restrict__ mean)
{
    for (int i = threadIdx.x; i < 4 * ny; i += blockDim.x) {
        const int f = i / ny, j = i - f * ny;
        const double m = mean_sum[i] / mean_count;
        mean[i] = mirror ? 0.5 * (m + (f == 1 ? -1.0 : 1.0) * (mean_sum[f * ny + ny - 1 - j] / mean_count)) : m;
    }
    __syncthreads();
    if (mirror)
        for (int i = threadIdx.x; i < 4 * ny; i += blockDim.x) mean_sum[i] = mean[i] * mean_count;
}

// ------------------------------------------- profiles from the raw sums
// prof[PR_*][y]: U and U' from the mean, the one-point averages from the
// products pass and eps = nu * (Parseval sum) / count.
__global__ void k_profiles(const double* __restrict__ mean_sum, double mean_count,
                           const double* __restrict__ stats, double snap_count, long long plane_points,
                           double nu, int mirror, const double* __restrict__ fdw, const int* __restrict__ fdl0,
                           int ny, double* __restrict__ prof)
{
    int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= ny) return;
    double dU = 0.0;
    for (int l = 0; l < 5; ++l) dU += fdw[5 * y + l] * (mean_sum[fdl0[y] + l] / mean_count);
    prof[PR_U * ny + y] = mean_sum[y] / mean_count;
    prof[PR_DU * ny + y] = dU;
    prof[PR_V * ny + y] = mean_sum[ny + y] / mean_count;
    prof[PR_W * ny + y] = mean_sum[2 * ny + y] / mean_count;
    prof[PR_P * ny + y] = mean_sum[3 * ny + y] / mean_count;
    // physical-space sums: over snapshots and the nx * nz plane points
    // with mirror sampling each statistic is the mean over the snapshots and
    // their mirror images, whose value at y is the snapshot's at ny - 1 - y
    // with the sign of v applied (odd in v: uv, pv, qv)
    const int ym = ny - 1 - y;
    auto st = [&](int s, double parity) {
        const double a = stats[s * ny + y];
        return mirror ? 0.5 * (a + parity * stats[s * ny + ym]) : a;
    };
    const double inv = 1.0 / (snap_count * (double)plane_points);
    prof[PR_Q * ny + y] = st(S_Q, 1.0) * inv;
    prof[PR_UV * ny + y] = st(S_UV, -1.0) * inv;
    prof[PR_PV * ny + y] = st(S_PV, -1.0) * inv;
    prof[PR_QU * ny + y] = st(S_QU, 1.0) * inv;
    prof[PR_QV * ny + y] = st(S_QV, -1.0) * inv;
    prof[PR_QW * ny + y] = st(S_QW, 1.0) * inv;
    // Parseval sums are already plane means: divide by the snapshot count only
    prof[PR_EPS * ny + y] = nu * st(S_EPS, 1.0) / snap_count;
}

}  // namespace gke
