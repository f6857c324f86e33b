/*
 * gke1h.h -- C ABI of the GKE evaluator for flows with ONE homogeneous
 * direction.
 *
 * Method: Gatti, Remigi, Chiarini, Cimarelli, Quadrio, "An efficient
 * numerical method for the Generalised Kolmogorov Equation".  The paper
 * builds its method for the plane channel (two homogeneous directions) and
 * notes in its conclusions (Sec. 5) that it carries over to flows with one
 * homogeneous direction, the extra inhomogeneous direction being handled like
 * the wall-normal one.  Here x is homogeneous and periodic; y and z are both
 * inhomogeneous, each on its own grid (a straight duct, for instance).  Every
 * GKE term is again a sum of two-point correlations plus one-point moments
 * (Sec. 3.1, Eq. 7); each correlation over x is the inverse Fourier transform
 * of a product of x-Fourier coefficients (Parseval, Eq. 8-9), summed over the
 * snapshots (Step 2), for every pair of cross-section points; the y and z
 * derivatives are 5-point finite differences in Y1, Y2 and in Z1, Z2 (Step 3,
 * Eq. 10-11, applied to both directions).
 *
 * Conventions
 *   - Grid: nx points over the period Lx; y[ny] and z[nz], each strictly
 *     increasing (ends included, no ghost nodes).  A cross-section point is
 *     p = iy nz + iz, P = ny nz points.
 *   - Input (complex128, re/im interleaved, host or device):
 *       fields[nsnap][4][ny][nz][nx/2 + 1]   u, v, w, p (mean included),
 *     forward-normalised over x only: a_hat(m) = 1/nx sum_x a(x) e^{-2 pi i m x / nx}
 *     (numpy/torch rfft(a, norm="forward") over the last axis).
 *   - Pairs: the npair = P (P + 1) / 2 ordered pairs (p1, p2), p1 <= p2,
 *     row-major (p1 outer).  Terms at p1 > p2 follow by r-inversion: A,
 *     psi_y, psi_z, xi and the residual are even, Phi_x, Phi_y, Phi_z odd
 *     under (p1, p2, r_x) -> (p2, p1, -r_x).
 *   - Separations: m_x in [0, nx), r_x = m_x Lx / nx (periodic).
 *   - Output terms (double on GKE_PREC_F64 plans, float on GKE_PREC_F32 plans;
 *     host or device):
 *       terms[GKE1H_NTERM][npair][nx]
 *     A = <du_i du_i>, then the fluxes in the space of scales
 *       Phi_k = <du_i du_i du_k> + A dU_k - 2 nu dA/dr_k         (k = x, y, z)
 *     the fluxes in physical space
 *       psi_k = <u_k* du_i du_i> + A U_k* + 2 <dp du_k> - (nu/2) dA/dX_k   (k = y, z)
 *     the source
 *       xi = sum_{i; k = y, z} [-2 <du_i du_k> (d_k U_i)* - 2 <du_i u_k*> d(d_k U_i)] - 4 eps*
 *     and the residual dPhi_x/dr_x + dPhi_y/dr_y + dPhi_z/dr_z + dpsi_y/dY + dpsi_z/dZ - xi
 *     (Sec. 2, Eq. 3-6 written for U_i(y, z): the channel's terms when the
 *     flow does not depend on z and U = (U(y), 0, 0), psi_y being its phi).
 *     Increments between (x, p1) and (x + r_x, p2); * is the mean of the two
 *     points; dU_k = U_k(p2) - U_k(p1); eps = nu <d_j u_i d_j u_i>.  r_x
 *     derivatives are spectral (signed wavenumber, 0 at the Nyquist index);
 *     r_y, Y and r_z, Z derivatives use the 5-point stencil of each grid
 *     (weights of gke_fd_weights; d/dr_y = (d_Y2 - d_Y1)/2, d/dY = d_Y1 + d_Y2).
 *   - Profiles (double [GKE1H_NPROF][P], optional): the mean of u, v, w, p over
 *     x and snapshots, the six mean-velocity gradients d_y U, d_z U, d_y V,
 *     d_z V, d_y W, d_z W (stencils), and eps.
 *   - Precision: FP64 throughout (GKE_PREC_F64), or the FP32 variant
 *     (GKE_PREC_F32; desc.precision).
 *   - Stream: every call is asynchronous on the plan's stream unless an
 *     argument is in host memory (then it returns after the last copy).
 */
#ifndef GKE1H_H
#define GKE1H_H

#include "gke.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gke1h_plan_s* gke1h_plan_t;

enum { GKE1H_TERM_A = 0, GKE1H_TERM_PHI_X, GKE1H_TERM_PHI_Y, GKE1H_TERM_PHI_Z, GKE1H_TERM_PSI_Y,
       GKE1H_TERM_PSI_Z, GKE1H_TERM_XI, GKE1H_TERM_RESIDUAL, GKE1H_NTERM };

enum { GKE1H_PROF_U = 0, GKE1H_PROF_V, GKE1H_PROF_W, GKE1H_PROF_P, GKE1H_PROF_DUDY, GKE1H_PROF_DUDZ,
       GKE1H_PROF_DVDY, GKE1H_PROF_DVDZ, GKE1H_PROF_DWDY, GKE1H_PROF_DWDZ, GKE1H_PROF_EPS, GKE1H_NPROF };

typedef struct {
    int nx;                /* homogeneous direction: 2^a or 3 * 2^a in [8, 512]          */
    int ny, nz;            /* inhomogeneous grids, each >= 5                               */
    double Lx;             /* period in x (> 0)                                            */
    double nu;             /* kinematic viscosity (> 0)                                    */
    const double* y;       /* host pointer, y[ny], strictly increasing; copied              */
    const double* z;       /* host pointer, z[nz], strictly increasing; copied              */
    int max_snap;          /* largest nsnap of any gke1h_compute call (sizes workspaces)  */
    int precision;         /* GKE_PREC_F64, or GKE_PREC_F32: operands, correlations, term
                              spectra, transforms and stencils in FP32 (means, products and
                              one-point sums stay FP64); GKE_PREC_BF16X3: GKE_ERR_UNSUPPORTED */
} gke1h_desc;

/* Create a plan: validates the descriptor (GKE_ERR_ARG on bad sizes, grids or
 * NULL pointers; GKE_ERR_UNSUPPORTED on nx outside the list above), computes
 * the stencil weights and twiddles on the host and allocates every
 * workspace on the current device (about c (8 npair + 11 max_snap P)
 * (nx/2 + 1) bytes, c = 16 on GKE_PREC_F64 plans and 8 on GKE_PREC_F32;
 * GKE_ERR_OOM if the device has not that much free).
 * stream: a cudaStream_t (NULL = legacy default stream).  Nothing is
 * allocated later except a staging buffer of the terms (8 or 4 bytes x
 * GKE1H_NTERM npair nx) on the first call with host-memory terms.           */
gke_status gke1h_plan(const gke1h_desc* desc, void* stream, gke1h_plan_t* out);

/* One full evaluation over nsnap snapshots (1 <= nsnap <= max_snap): the
 * mean over x and snapshots, the fluctuations and their in-plane products,
 * the snapshot sums of the x-correlations of every pair with the terms
 * formed per wavenumber, the inverse transforms in x and the stencils.
 * fields, terms and profiles (may be NULL) in host or device memory (layouts
 * above).  GKE_ERR_NONFINITE if the input holds a NaN or Inf (outputs are
 * then undefined).                                                          */
gke_status gke1h_compute(gke1h_plan_t plan, const void* fields, int nsnap, void* terms, double* profiles);

/* Number of pairs, P (P + 1) / 2.                                           */
long long gke1h_npair(gke1h_plan_t plan);

/* Host utility (no plan, no GPU): the labels of the npair = P (P + 1) / 2
 * output pairs of grids y[ny], z[nz], in output order (p1 <= p2, p1
 * outer): the point indices p1[], p2[] (p = iy nz + iz) and the coordinates
 * Y1 = y[p1 / nz], Z1 = z[p1 % nz], Y2, Z2.  Any output may be NULL.
 * Returns npair, or -1 on bad arguments (NULL grids, ny or nz < 1).          */
long long gke1h_pair_labels(int ny, int nz, const double* y, const double* z, int* p1, int* p2, double* Y1,
                            double* Z1, double* Y2, double* Z2);

/* Stage timing as for gke_set_timing / gke_stage_times (ms[GKE_NSTAGE]:
 * mean, products and one-point sums, correlate (with the per-pair term
 * spectra), combine (always 0), inverse transforms, stencils).             */
gke_status gke1h_set_timing(gke1h_plan_t plan, int on);
gke_status gke1h_stage_times(gke1h_plan_t plan, double* ms);
long long gke1h_launch_count(gke1h_plan_t plan);

/* Message of the last failed call on this plan (plan == NULL: the last
 * gke1h_plan failure of the calling thread).                                */
const char* gke1h_last_error(gke1h_plan_t plan);

/* Free every resource of the plan (synchronises its stream).  NULL is a no-op. */
void gke1h_destroy(gke1h_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* GKE1H_H */
