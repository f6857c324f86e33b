// gke_terms.cu -- from per-wavenumber spectral sums to the GKE terms.
//
// Inverse transform (Sec. 3.1, Eq. 9) of the spectra each term needs, the
// one-point parts of the correlation expansion (Eq. 7), and the Step-3
// finite-difference derivatives in Y1 / Y2 (Sec. 3.2, Eq. 10-11) with values
// across the diagonal recovered by r-inversion (Sec. 3.3).
//
// With S0 = D, S1 = E + E^H, S2 = E^H - E, S3 = F + F^H, S4 = Gx - Gx^H,
// S5 = Gy - Gy^H, S6 = Gz - Gz^H, S7 = H + H^H (X^H(y, y') = conj X(y', y),
// Gy = QV + X2, H = QV - X2 with X2 the stored 2 sum_i conj(u_i v) u_i),
// every term is one inverse transform of a
// linear combination of the S_n plus a part that depends only on (Y1, Y2):
//   A     = F^-1[-2 S0]                                 + <q>1 + <q>2
//   Phi_x = F^-1[S4 + (-2 dU + 4 i nu kx) S0]           + <qu>2 - <qu>1 + dU (<q>1 + <q>2)
//   Phi_y = F^-1[S5]                                    + <qv>2 - <qv>1     (+ FD part)
//   Phi_z = F^-1[S6 + 4 i nu kz S0]                     + <qw>2 - <qw>1
//   phi   = F^-1[S7 / 2 - 2 S3]                         + (<qv>1 + <qv>2)/2 + 2 (<pv>1 + <pv>2)  (+ FD)
//   xi    = F^-1[2 U'* S1 - dU' S2]                     - 2 U'* (<uv>1 + <uv>2) - dU' (<uv>2 - <uv>1) - 2 (eps1 + eps2)
//   res   = F^-1[i kx S4 + i kz S6 - 2 i dU kx S0 - 4 nu |k|^2 S0] - xi   (+ FD parts)
// (q = u_i u_i, dU = U(Y2) - U(Y1), U'* = (U'(Y1) + U'(Y2))/2, dU' = U'(Y2) - U'(Y1)).
#include "gke_common.cuh"
#include "gke_kernels.h"

namespace gke {

#define TWO_PI 6.283185307179586476925286766559

// per-wavenumber combination of the spectral sums for one pair
__device__ __forceinline__ void combos(const zd* __restrict__ acc_sq, const zd* __restrict__ acc_D,
                                       long long p, int i1, int i2, int ny, int Nk, long long k,
                                       double kx, double kz, const PairCoef& pc, zd T[NTERM])
{
    const long long sq = (long long)ny * ny;
    const long long o12 = ((long long)i1 * ny + i2) * Nk + k, o21 = ((long long)i2 * ny + i1) * Nk + k;
    const double ic = pc.inv_count;
    zd S0 = ic * acc_D[p * Nk + k];
    zd E12 = acc_sq[J_E * sq * Nk + o12], E21 = conj(acc_sq[J_E * sq * Nk + o21]);
    zd F12 = acc_sq[J_F * sq * Nk + o12], F21 = conj(acc_sq[J_F * sq * Nk + o21]);
    zd Gx12 = acc_sq[J_GX * sq * Nk + o12], Gx21 = conj(acc_sq[J_GX * sq * Nk + o21]);
    zd Gz12 = acc_sq[J_GZ * sq * Nk + o12], Gz21 = conj(acc_sq[J_GZ * sq * Nk + o21]);
    zd Q12 = acc_sq[J_QV * sq * Nk + o12], Q21 = conj(acc_sq[J_QV * sq * Nk + o21]);
    zd X12 = acc_sq[J_X * sq * Nk + o12], X21 = conj(acc_sq[J_X * sq * Nk + o21]);
    zd S1 = ic * (E12 + E21), S2 = ic * (E21 - E12), S3 = ic * (F12 + F21);
    zd S4 = ic * (Gx12 - Gx21), S6 = ic * (Gz12 - Gz21);
    zd S5 = ic * ((Q12 + X12) - (Q21 + X21));
    zd S7 = ic * ((Q12 - X12) + (Q21 - X21));
    const double nu = pc.nu;
    T[T_A] = -2.0 * S0;
    T[T_PHIX] = S4 + (-2.0 * pc.dU) * S0 + (4.0 * nu * kx) * mul_i(S0);
    T[T_PHIY] = S5;
    T[T_PHIZ] = S6 + (4.0 * nu * kz) * mul_i(S0);
    T[T_PHI] = 0.5 * S7 - 2.0 * S3;
    T[T_XI] = (2.0 * pc.Upm) * S1 - pc.dUp * S2;
    T[T_RES] = kx * mul_i(S4) + kz * mul_i(S6) + (-2.0 * pc.dU * kx) * mul_i(S0)
             + (-4.0 * nu * (kx * kx + kz * kz)) * S0 - T[T_XI];
}

__device__ __forceinline__ PairCoef pair_coef(const double* __restrict__ prof, int ny, int i1, int i2,
                                              double nu, double inv_count)
{
    PairCoef pc;
    pc.dU = prof[PR_U * ny + i2] - prof[PR_U * ny + i1];
    pc.Upm = 0.5 * (prof[PR_DU * ny + i1] + prof[PR_DU * ny + i2]);
    pc.dUp = prof[PR_DU * ny + i2] - prof[PR_DU * ny + i1];
    pc.nu = nu;
    pc.inv_count = inv_count;
    return pc;
}

// -------------------------- column pass: combine + inverse transform along z
// W[pl][t][z][kx] = sum_kz T_t(kz, kx) e^{+i kz z}, pl = local pair index.
// CTA = CW kx columns of one pair; shared memory NTERM * CW * nz complex.
__global__ void k_terms_colpass(const zd* __restrict__ acc_sq, const zd* __restrict__ acc_D,
                                const int* __restrict__ pair_i, long long pair0, int ny, int nz, int nx,
                                int CW, double Lx, double Lz, double nu, double inv_count,
                                const double* __restrict__ prof, const zd* __restrict__ tw_z,
                                zd* __restrict__ W)
{
    extern __shared__ zd sh_tc[];
    const int nxh = nx / 2 + 1, Nk = nz * nxh, lg = ilog2(nz);
    const int kx0 = blockIdx.x * CW;
    const long long pl = blockIdx.y, p = pair0 + pl;
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    const PairCoef pc = pair_coef(prof, ny, i1, i2, nu, inv_count);
    for (int t = threadIdx.x; t < CW * nz; t += blockDim.x) {
        int c = t % CW, kz_i = t / CW, kx_i = kx0 + c;
        zd T[NTERM];
        if (kx_i < nxh) {
            double kx = TWO_PI * signed_bin(kx_i, nx) / Lx;
            double kz = TWO_PI * signed_bin(kz_i, nz) / Lz;
            combos(acc_sq, acc_D, p, i1, i2, ny, Nk, (long long)kz_i * nxh + kx_i, kx, kz, pc, T);
        } else {
            for (int q = 0; q < NTERM; ++q) T[q] = mk(0.0, 0.0);
        }
        int br = bitrev(kz_i, lg);
        for (int q = 0; q < NTERM; ++q) sh_tc[(q * CW + c) * nz + br] = T[q];
    }
    fft_radix2_block(sh_tc, nz, NTERM * CW, lg, tw_z, +1);
    for (int t = threadIdx.x; t < NTERM * CW * nz; t += blockDim.x) {
        int c = t % CW, rem = t / CW, z = rem % nz, q = rem / nz, kx_i = kx0 + c;
        if (kx_i < nxh) W[((pl * NTERM + q) * nz + z) * nxh + kx_i] = sh_tc[(q * CW + c) * nz + z];
    }
}

// ------------------------------ row pass: C2R along x + one-point parts
// terms[t][p][z][x] = sum_kx W[pl][t][z][kx] e^{+i kx x} + onepoint_t(Y1, Y2).
// Terms are transformed two at a time (t0 + i t1).  CTA = RZ rows of one pair;
// shared memory RZ * 4 * nx complex.
__global__ void k_terms_rowpass(const zd* __restrict__ W, const int* __restrict__ pair_i, long long pair0,
                                long long npair, int ny, int nz, int nx, int RZ,
                                const double* __restrict__ prof, const zd* __restrict__ tw_x,
                                double* __restrict__ terms)
{
    extern __shared__ zd sh_tr[];
    const int nxh = nx / 2 + 1, lg = ilog2(nx);
    const int z0 = blockIdx.x * RZ;
    const int nrow = min(RZ, nz - z0);
    const long long pl = blockIdx.y, p = pair0 + pl;
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    for (int t = threadIdx.x; t < nrow * 4 * nx; t += blockDim.x) {
        int r = t / (4 * nx), rem = t - r * 4 * nx, j = rem / nx, k = rem - j * nx;
        int z = z0 + r;
        int ta = 2 * j, tb = 2 * j + 1;
        const zd* wa = W + ((pl * NTERM + ta) * nz + z) * nxh;
        zd A, B = mk(0.0, 0.0);
        if (k < nxh) A = wa[k]; else A = conj(wa[nx - k]);
        if (tb < NTERM) {
            const zd* wb = W + ((pl * NTERM + tb) * nz + z) * nxh;
            if (k < nxh) B = wb[k]; else B = conj(wb[nx - k]);
        }
        if (k == 0 || 2 * k == nx) { A.y = 0.0; B.y = 0.0; }
        sh_tr[(r * 4 + j) * nx + bitrev(k, lg)] = mk(A.x - B.y, A.y + B.x);
    }
    fft_radix2_block(sh_tr, nx, 4 * nrow, lg, tw_x, +1);
    // one-point parts (Eq. 7): they depend on (Y1, Y2) only
    const double* pr = prof;
    double q1 = pr[PR_Q * ny + i1], q2 = pr[PR_Q * ny + i2];
    double uv1 = pr[PR_UV * ny + i1], uv2 = pr[PR_UV * ny + i2];
    double pv1 = pr[PR_PV * ny + i1], pv2 = pr[PR_PV * ny + i2];
    double qu1 = pr[PR_QU * ny + i1], qu2 = pr[PR_QU * ny + i2];
    double qv1 = pr[PR_QV * ny + i1], qv2 = pr[PR_QV * ny + i2];
    double qw1 = pr[PR_QW * ny + i1], qw2 = pr[PR_QW * ny + i2];
    double e1 = pr[PR_EPS * ny + i1], e2 = pr[PR_EPS * ny + i2];
    double dU = pr[PR_U * ny + i2] - pr[PR_U * ny + i1];
    double Upm = 0.5 * (pr[PR_DU * ny + i1] + pr[PR_DU * ny + i2]);
    double dUp = pr[PR_DU * ny + i2] - pr[PR_DU * ny + i1];
    double one[NTERM];
    one[T_A] = q1 + q2;
    one[T_PHIX] = (qu2 - qu1) + dU * (q1 + q2);
    one[T_PHIY] = qv2 - qv1;
    one[T_PHIZ] = qw2 - qw1;
    one[T_PHI] = 0.5 * (qv1 + qv2) + 2.0 * (pv1 + pv2);
    one[T_XI] = -2.0 * Upm * (uv1 + uv2) - dUp * (uv2 - uv1) - 2.0 * (e1 + e2);
    one[T_RES] = -one[T_XI];
    const long long N = (long long)nz * nx;
    for (int t = threadIdx.x; t < nrow * NTERM * nx; t += blockDim.x) {
        int r = t / (NTERM * nx), rem = t - r * NTERM * nx, q = rem / nx, x = rem - q * nx;
        zd v = sh_tr[(r * 4 + (q >> 1)) * nx + x];
        double val = ((q & 1) ? v.y : v.x) + one[q];
        terms[((long long)q * npair + p) * N + (long long)(z0 + r) * nx + x] = val;
    }
}

// ----------------------------------------------- Step 3 FD stencils
// value of term t at the ordered pair (a, b) and separation index rr, taken
// from the stored triangle a <= b, or by r-inversion (Sec. 3.3) with parity sg
__device__ __forceinline__ double tri_value(const double* __restrict__ term, int a, int b, int ny, int nz, int nx,
                                            int mz, int mx, double sg)
{
    const long long N = (long long)nz * nx;
    if (a <= b) return term[pair_index(a, b, ny) * N + (long long)mz * nx + mx];
    int mzn = (nz - mz) % nz, mxn = (nx - mx) % nx;
    return sg * term[pair_index(b, a, ny) * N + (long long)mzn * nx + mxn];
}

// pass 1: Phi_y -= 2 nu dA/dr_y, phi -= (nu/2) dA/dY, dA/dr_y = (d_Y2 - d_Y1) A / 2,
// dA/dY = (d_Y1 + d_Y2) A (Eq. 10-11).  A is even under r-inversion.
// grid: (ceil(nz*nx / blockDim), npair)
__global__ void k_stencil_A(double* __restrict__ terms, long long npair, const int* __restrict__ pair_i,
                            int ny, int nz, int nx, double nu, const double* __restrict__ fdw,
                            const int* __restrict__ fdl0)
{
    const long long N = (long long)nz * nx;
    const long long p = blockIdx.y;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int mz = (int)(e / nx), mx = (int)(e - (long long)mz * nx);
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    const double* A = terms + (long long)T_A * npair * N;
    double d1 = 0.0, d2 = 0.0;
    const int a1 = fdl0[i1], a2 = fdl0[i2];
    #pragma unroll
    for (int l = 0; l < 5; ++l) {
        d1 += fdw[5 * i1 + l] * tri_value(A, a1 + l, i2, ny, nz, nx, mz, mx, 1.0);
        d2 += fdw[5 * i2 + l] * tri_value(A, i1, a2 + l, ny, nz, nx, mz, mx, 1.0);
    }
    terms[((long long)T_PHIY * npair + p) * N + e] += -2.0 * nu * 0.5 * (d2 - d1);
    terms[((long long)T_PHI * npair + p) * N + e] += -0.5 * nu * (d1 + d2);
}

// pass 2: res += dPhi_y/dr_y + dphi/dY by the same stencil; Phi_y is odd and
// phi even under r-inversion.
__global__ void k_stencil_res(double* __restrict__ terms, long long npair, const int* __restrict__ pair_i,
                              int ny, int nz, int nx, const double* __restrict__ fdw,
                              const int* __restrict__ fdl0)
{
    const long long N = (long long)nz * nx;
    const long long p = blockIdx.y;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int mz = (int)(e / nx), mx = (int)(e - (long long)mz * nx);
    const int i1 = pair_i[2 * p], i2 = pair_i[2 * p + 1];
    const double* Py = terms + (long long)T_PHIY * npair * N;
    const double* Ph = terms + (long long)T_PHI * npair * N;
    double y1 = 0.0, y2 = 0.0, h1 = 0.0, h2 = 0.0;
    const int a1 = fdl0[i1], a2 = fdl0[i2];
    #pragma unroll
    for (int l = 0; l < 5; ++l) {
        double w1 = fdw[5 * i1 + l], w2 = fdw[5 * i2 + l];
        y1 += w1 * tri_value(Py, a1 + l, i2, ny, nz, nx, mz, mx, -1.0);
        y2 += w2 * tri_value(Py, i1, a2 + l, ny, nz, nx, mz, mx, -1.0);
        h1 += w1 * tri_value(Ph, a1 + l, i2, ny, nz, nx, mz, mx, 1.0);
        h2 += w2 * tri_value(Ph, i1, a2 + l, ny, nz, nx, mz, mx, 1.0);
    }
    terms[((long long)T_RES * npair + p) * N + e] += 0.5 * (y2 - y1) + (h1 + h2);
}

// ------------------------------------------- profiles from the raw sums
// prof[PR_*][y]: U and U' from the mean, the one-point averages from the
// products pass and eps = nu * (Parseval sum) / count.
__global__ void k_profiles(const double* __restrict__ mean_sum, double mean_count,
                           const double* __restrict__ stats, double snap_count, long long plane_points,
                           double nu, const double* __restrict__ fdw, const int* __restrict__ fdl0, int ny,
                           double* __restrict__ prof)
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
    const double inv = 1.0 / (snap_count * (double)plane_points);
    prof[PR_Q * ny + y] = stats[S_Q * ny + y] * inv;
    prof[PR_UV * ny + y] = stats[S_UV * ny + y] * inv;
    prof[PR_PV * ny + y] = stats[S_PV * ny + y] * inv;
    prof[PR_QU * ny + y] = stats[S_QU * ny + y] * inv;
    prof[PR_QV * ny + y] = stats[S_QV * ny + y] * inv;
    prof[PR_QW * ny + y] = stats[S_QW * ny + y] * inv;
    // Parseval sums are already plane means: divide by the snapshot count only
    prof[PR_EPS * ny + y] = nu * stats[S_EPS * ny + y] / snap_count;
}

}  // namespace gke
