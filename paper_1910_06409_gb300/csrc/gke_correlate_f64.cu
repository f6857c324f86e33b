// gke_correlate_f64.cu -- CUDA-core correlator, FP64 (plain path) and FP32.
//
// For every wavenumber k the paper's Parseval step (Sec. 3.1, Eq. 8-9) needs
// sums over snapshots of conj(a_hat(y, k)) b_hat(y', k) for the field pairs
// of the expansion (Eq. 7).  Per k these are small dense complex products
//   S(y, y') = sum_t sum_s conj(A_t[s][y]) B_t[s][y']
// over the operand blocks Xop[f][k][s][y].  The contractions ("jobs"):
//   D   = sum_i conj(u_i) u_i                    (Hermitian: pairs y <= y')
//   E   = conj(u) v,   F = conj(p) v
//   Gx  = conj(q) u + 2 [conj(uu) u + conj(uv) v + conj(uw) w]
//   QV  = conj(q) v,   X2 = 2 [conj(uv) u + conj(vv) v + conj(vw) w]
//   Gz  = conj(q) w + 2 [conj(uw) u + conj(vw) v + conj(ww) w]
// (the operand blocks of uu .. vw already hold the factor 2: k_col_forward)
// (the y-flux triple terms are QV + X2 and QV - X2, formed later).
//
// CTA = one wavenumber of a chunk and one job; it walks tiles of (y, y'), each thread
// holding an RB x RB block of complex accumulators, and writes the batch's
// contraction to raw (8 x 8 pair-block layout, raw_index; D: y <= y' only).
// FP64: DFMA bound.  FP32: the same sums in FFMA with FP32 accumulation.  When ny leaves a thin remainder past the last full tile (the
// Chebyshev grids ny = 32 m + 1 leave one wall row), that remainder is done
// as row and column strips, one (y, y') per thread, instead of as mostly empty
// padded tiles (which cost half as much again as the useful work at ny = 129).
#include "gke_common.cuh"
#include "gke_kernels.h"

namespace gke {

struct JobDesc { int nterm; int fa[4]; int fb[4]; };

__constant__ JobDesc c_jobs[NJSQ + 1];   // index NJSQ = D

void upload_jobs(cudaStream_t st)
{
    JobDesc h[NJSQ + 1] = {
        /* E  */ {1, {F_U, 0, 0, 0}, {F_V, 0, 0, 0}},
        /* F  */ {1, {F_P, 0, 0, 0}, {F_V, 0, 0, 0}},
        /* GX */ {4, {F_Q, F_UU, F_UV, F_UW}, {F_U, F_U, F_V, F_W}},
        /* QV */ {1, {F_Q, 0, 0, 0}, {F_V, 0, 0, 0}},
        /* X2 */ {3, {F_UV, F_VV, F_VW, 0}, {F_U, F_V, F_W, 0}},
        /* GZ */ {4, {F_Q, F_UW, F_VW, F_WW}, {F_W, F_U, F_V, F_W}},
        /* D  */ {3, {F_U, F_V, F_W, 0}, {F_U, F_V, F_W, 0}},
    };
    cudaMemcpyToSymbolAsync(c_jobs, h, sizeof(h), 0, cudaMemcpyHostToDevice, st);
}

// acc += conj(a) b as four fused multiply-adds (written out: the plain
// expression would contract to a multiply, an FMA and an add per component)
template <typename T>
__device__ __forceinline__ void cmac_conj(cplx<T>& acc, const cplx<T> a, const cplx<T> b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

#define SCH 8       // snapshots per shared-memory chunk
#define STRIP_MAX 4 // widest remainder done as strips

// T = double: RB = 2 (32 x 32 tiles, DFMA bound); T = float: RB = 4 (64 x 64
// tiles, so each thread does 4 FFMA per shared-memory load)
// the contractions one launch runs (a term mask may leave some out)
struct JobList { int n; int j[NJOB]; };

template <typename T, int RB>
__global__ void __launch_bounds__(256)
k_correlate(const cplx<T>* __restrict__ Xop, int ns, int ny, int Nk, int k0, int Kc, JobList jl,
            cplx<T>* __restrict__ raw)
{
    typedef cplx<T> C;
    constexpr int CT = 16 * RB;     // tile edge
    __shared__ C As[SCH][CT];
    __shared__ C Bs[SCH][CT];
    const int kl = blockIdx.x, k = k0 + kl, job = jl.j[blockIdx.y];    // chunk-local and global wavenumber
    const bool herm = (job == NJSQ);
    const JobDesc& jd = c_jobs[job];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int nfull = ny / CT, rem = ny - nfull * CT;
    const bool strips = nfull > 0 && rem > 0 && rem <= STRIP_MAX;
    const int nt = strips ? nfull : (ny + CT - 1) / CT;
    for (int tb0 = 0; tb0 < nt; ++tb0) {
        for (int tb1 = herm ? tb0 : 0; tb1 < nt; ++tb1) {
            const int y0 = tb0 * CT, y1 = tb1 * CT;
            C acc[RB][RB];
            #pragma unroll
            for (int a = 0; a < RB; ++a)
                #pragma unroll
                for (int b = 0; b < RB; ++b) acc[a][b] = mk((T)0, (T)0);
            for (int t = 0; t < jd.nterm; ++t) {
                const C* A = Xop + ((long long)jd.fa[t] * Nk + k) * ns * ny;
                const C* B = Xop + ((long long)jd.fb[t] * Nk + k) * ns * ny;
                for (int s0 = 0; s0 < ns; s0 += SCH) {
                    __syncthreads();
                    for (int e = threadIdx.x; e < SCH * CT; e += blockDim.x) {
                        int ss = e / CT, yy = e - ss * CT;
                        int s = s0 + ss;
                        C va = mk((T)0, (T)0), vb = mk((T)0, (T)0);
                        if (s < ns && y0 + yy < ny) va = A[(long long)s * ny + y0 + yy];
                        if (s < ns && y1 + yy < ny) vb = B[(long long)s * ny + y1 + yy];
                        As[ss][yy] = va;
                        Bs[ss][yy] = vb;
                    }
                    __syncthreads();
                    #pragma unroll
                    for (int ss = 0; ss < SCH; ++ss) {
                        C a[RB], bb[RB];
                        #pragma unroll
                        for (int i = 0; i < RB; ++i) { a[i] = As[ss][ty + 16 * i]; bb[i] = Bs[ss][tx + 16 * i]; }
                        #pragma unroll
                        for (int i = 0; i < RB; ++i)
                            #pragma unroll
                            for (int j = 0; j < RB; ++j) cmac_conj(acc[i][j], a[i], bb[j]);
                    }
                }
            }
            #pragma unroll
            for (int a = 0; a < RB; ++a)
                #pragma unroll
                for (int b = 0; b < RB; ++b) {
                    int y = y0 + ty + 16 * a, yp = y1 + tx + 16 * b;
                    if (y >= ny || yp >= ny) continue;
                    if (herm && yp < y) continue;
                    raw[raw_index(job, kl, y, yp, Kc, (ny + 7) / 8)] = acc[a][b];
                }
        }
    }
    if (!strips) return;
    // remainder strips: rows y >= cov against every y' (D: y' >= y), then
    // columns y' >= cov against y < cov
    const int cov = nfull * CT;
    const int nrow = rem * ny, ncol = cov * rem;
    for (int e = threadIdx.x; e < nrow + ncol; e += blockDim.x) {
        int y, yp;
        if (e < nrow) {
            y = cov + e / ny;
            yp = e - (y - cov) * ny;
            if (herm && yp < y) continue;
        } else {
            const int f = e - nrow;
            y = f / rem;
            yp = cov + (f - y * rem);
        }
        C acc = mk((T)0, (T)0);
        for (int t = 0; t < jd.nterm; ++t) {
            const C* A = Xop + ((long long)jd.fa[t] * Nk + k) * ns * ny;
            const C* B = Xop + ((long long)jd.fb[t] * Nk + k) * ns * ny;
            for (int s = 0; s < ns; ++s) cmac_conj(acc, A[(long long)s * ny + y], B[(long long)s * ny + yp]);
        }
        raw[raw_index(job, kl, y, yp, Kc, (ny + 7) / 8)] = acc;
    }
}

// wavenumbers [k0, k0 + Kc) of Nk; raw holds the chunk (raw_index with Kc)
void correlate_launch(bool fp32, const void* Xop, int ns, int ny, int Nk, int k0, int Kc, void* raw, unsigned jobs,
                      cudaStream_t st)
{
    JobList jl{};
    for (int j = 0; j < NJOB; ++j)
        if ((jobs >> j) & 1u) jl.j[jl.n++] = j;
    if (jl.n == 0) return;
    if (fp32)
        k_correlate<float, 4><<<dim3(Kc, jl.n), 256, 0, st>>>((const zf*)Xop, ns, ny, Nk, k0, Kc, jl, (zf*)raw);
    else
        k_correlate<double, 2><<<dim3(Kc, jl.n), 256, 0, st>>>((const zd*)Xop, ns, ny, Nk, k0, Kc, jl, (zd*)raw);
}

}  // namespace gke
