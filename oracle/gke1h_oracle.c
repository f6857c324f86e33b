/*
 * gke1h_oracle.c -- CPU oracle for the GKE of a flow with ONE homogeneous
 * direction.
 *
 * TEST INFRASTRUCTURE ONLY.  The plain, slow reference the CUDA path of the
 * one-homogeneous-direction variant is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header, table or helper with
 * the CUDA path.
 *
 * What it computes.  The paper (Gatti et al., Sec. 5) notes that its method
 * carries over to flows with a single homogeneous direction, the second
 * inhomogeneous direction being handled like the wall-normal direction of
 * the channel.  Here x is homogeneous (periodic, length Lx) and both y and z
 * are inhomogeneous, each sampled on its own grid.  A point of the cross
 * section is p = (iy, iz), linear index p = iy nz + iz.  For two points
 * p1 = (Y1, Z1), p2 = (Y2, Z2) and a separation m_x (r_x = m_x Lx / nx),
 * x' = x + r_x:
 *     delta f = f(x', p2) - f(x, p1),   f* = (f(x, p1) + f(x', p2)) / 2,
 * averaged over x and snapshots only (the one homogeneous direction):
 *     A    = <du_i du_i>
 *     B_k  = <du_i du_i du_k>,  k = x, y, z
 *     C_k  = <u_k* du_i du_i>,  k = y, z
 *     P_k  = <dp du_k>,         k = y, z       (rho = 1)
 *     Q_ik = <du_i du_k>,       i = x, y, z;  k = y, z
 *     R_ik = <du_i u_k*>,       i = x, y, z;  k = y, z
 *     GxA  = dA/dr_x = <2 du_i (d_x u_i)(x', p2)>  (spectral d_x, Nyquist 0)
 * the derivatives in Y1, Y2, Z1, Z2 by the 5-point stencil of each grid
 * (Step 3, Eq. 10-11, applied to y and to z alike),
 *     d/dr_y = (d_Y2 - d_Y1) / 2,  d/dY = d_Y1 + d_Y2,  and the same in z,
 * and the terms of the GKE written as in Sec. 2 with the mean velocity
 * U_i(y, z) (all three components; the channel has only U(y)):
 *     Phi_x = B_x + A dU_x - 2 nu GxA                         (Eq. 4)
 *     Phi_y = B_y + A dU_y - 2 nu dA/dr_y
 *     Phi_z = B_z + A dU_z - 2 nu dA/dr_z
 *     psi_y = C_y + A U_y* + 2 P_y - (nu/2) dA/dY             (Eq. 5)
 *     psi_z = C_z + A U_z* + 2 P_z - (nu/2) dA/dZ
 *     xi    = sum_{i, k} [-2 Q_ik (d_k U_i)* - 2 R_ik d(d_k U_i)] - 4 eps*   (Eq. 6)
 *     res   = dPhi_x/dr_x + dPhi_y/dr_y + dPhi_z/dr_z + dpsi_y/dY + dpsi_z/dZ - xi
 * with dU_k = U_k(p2) - U_k(p1), U_k* their mean, d_k U_i by the stencil of
 * the k grid, eps = nu <d_j u_i d_j u_i> (x spectral, y and z by the
 * stencils).  For U = (U(y), 0, 0) and fields that do not depend on z these
 * are the channel's terms (psi_y is its phi).  The mean-flow terms follow
 * the general inhomogeneous form of the equation: advection by the mean in
 * the space of scales (A dU_k) and in physical space (A U_k*), production by
 * every mean-velocity gradient.
 *
 * Readings: averages are means over grid points and snapshots; each grid's
 * stencil is the 5-point first-derivative formula exact on polynomials of
 * degree <= 4 (window j-2..j+2, shifted to 0..4 / n-5..n-1 next to an end),
 * its weights from the 5x5 moment (Vandermonde) system; every ordered pair
 * is computed directly, so the stencils never need values from across the
 * diagonal.  Fluctuations are taken about the mean over x and snapshots.
 *
 * Layouts (C order), P = ny nz:
 *   phys  double [ns][4][ny][nz][nx]   u, v, w, p including the mean
 *   comp  double [NCOMP][P][P][nx]     ordered pairs (p1, p2), then m_x
 *   terms double [NTERM][P][P][nx]
 *   prof  double [NPROF][P]
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { C_A = 0, C_BX, C_BY, C_BZ, C_CY, C_CZ, C_PY, C_PZ,
       C_Q,                      /* Q_ik at C_Q + 3 (k - 1) + i: xy yy zy xz yz zz */
       C_R = C_Q + 6,            /* R_ik likewise                                   */
       C_GXA = C_R + 6, C_DY1, C_DY2, C_DZ1, C_DZ2, NCOMP };
enum { T_A = 0, T_PHIX, T_PHIY, T_PHIZ, T_PSIY, T_PSIZ, T_XI, T_RES, NTERM };
enum { P_U = 0, P_V, P_W, P_P,
       P_G,                      /* d_k U_i at P_G + 2 i + (k - 1): dU/dy dU/dz dV/dy dV/dz dW/dy dW/dz */
       P_EPS = P_G + 6, NPROF };

int oracle1h_ncomp(void) { return NCOMP; }
int oracle1h_nterm(void) { return NTERM; }
int oracle1h_nprof(void) { return NPROF; }

/* 5-point first-derivative weights at row j of the grid g[n] (moment system,
 * Gaussian elimination with partial pivoting); returns the window start.  */
static int fd5(const double *g, int n, int j, double *w)
{
    int l0 = j - 2;
    if (l0 < 0) l0 = 0;
    if (l0 > n - 5) l0 = n - 5;
    double t[5], h = 0.0;
    for (int l = 0; l < 5; ++l) {
        t[l] = g[l0 + l] - g[j];
        if (fabs(t[l]) > h) h = fabs(t[l]);
    }
    double M[5][6];
    for (int p = 0; p < 5; ++p) {
        for (int l = 0; l < 5; ++l) M[p][l] = pow(t[l] / h, p);
        M[p][5] = (p == 1) ? 1.0 : 0.0;
    }
    for (int c = 0; c < 5; ++c) {
        int piv = c;
        for (int r = c + 1; r < 5; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 6; ++k) { double tmp = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = tmp; }
        for (int r = c + 1; r < 5; ++r) {
            double f = M[r][c] / M[c][c];
            for (int k = c; k < 6; ++k) M[r][k] -= f * M[c][k];
        }
    }
    double s[5];
    for (int r = 4; r >= 0; --r) {
        double acc = M[r][5];
        for (int k = r + 1; k < 5; ++k) acc -= M[r][k] * s[k];
        s[r] = acc / M[r][r];
    }
    for (int l = 0; l < 5; ++l) w[l] = s[l] / h;
    return l0;
}

/* d/dx of a real periodic sequence f[0..n) (period L) by naive DFT: multiply
 * the coefficient of index m by i k_m, k_m = 2 pi m' / L with m' the signed
 * index, 0 at m = n/2.  cs[j], sn[j] = cos, sin of 2 pi j / n.            */
static void dft_deriv(const double *f, double *df, int n, double L, const double *cs, const double *sn)
{
    double *re = (double *)malloc(sizeof(double) * 2 * n);
    double *im = re + n;
    for (int m = 0; m < n; ++m) {
        double ar = 0.0, ai = 0.0;
        for (int x = 0; x < n; ++x) {
            int ph = (int)(((long)m * x) % n);
            ar += f[x] * cs[ph];
            ai -= f[x] * sn[ph];
        }
        ar /= n; ai /= n;
        int ms = (m < n / 2) ? m : m - n;
        if (2 * m == n) ms = 0;
        double k = 2.0 * M_PI * ms / L;
        re[m] = -k * ai;
        im[m] = k * ar;
    }
    for (int x = 0; x < n; ++x) {
        double acc = 0.0;
        for (int m = 0; m < n; ++m) {
            int ph = (int)(((long)m * x) % n);
            acc += re[m] * cs[ph] - im[m] * sn[ph];
        }
        df[x] = acc;
    }
    free(re);
}

typedef struct {
    int ns, nx, ny, nz, P;
    double Lx, nu;
    double *fl;          /* fluctuations [ns][4][P][nx] */
    double *dx;          /* d_x u_i [ns][3][P][nx] */
    double *prof;        /* [NPROF][P] */
    double *cs, *sn;     /* cos, sin of 2 pi j / nx */
    double *wy, *wz;     /* [ny][5], [nz][5] */
    int *ly, *lz;        /* window starts */
} ctx1h;

#define FL(c, s, f, p) ((c)->fl + ((((long)(s) * 4 + (f)) * (c)->P + (p)) * (c)->nx))
#define DXU(c, s, i, p) ((c)->dx + ((((long)(s) * 3 + (i)) * (c)->P + (p)) * (c)->nx))

static void ctx_free(ctx1h *c)
{
    free(c->fl); free(c->dx); free(c->prof); free(c->wy); free(c->wz); free(c->ly); free(c->lz); free(c->cs);
}

static int ctx_init(ctx1h *c, const double *phys, int ns, int nx, int ny, int nz, const double *y,
                    const double *z, double Lx, double nu)
{
    memset(c, 0, sizeof(*c));
    if (ns < 1 || nx < 2 || ny < 5 || nz < 5) return -1;
    c->ns = ns; c->nx = nx; c->ny = ny; c->nz = nz; c->P = ny * nz;
    c->Lx = Lx; c->nu = nu;
    long P = c->P;
    c->fl = (double *)malloc(sizeof(double) * ns * 4 * P * nx);
    c->dx = (double *)malloc(sizeof(double) * ns * 3 * P * nx);
    c->prof = (double *)calloc(NPROF * P, sizeof(double));
    c->wy = (double *)malloc(sizeof(double) * 5 * ny);
    c->wz = (double *)malloc(sizeof(double) * 5 * nz);
    c->ly = (int *)malloc(sizeof(int) * ny);
    c->lz = (int *)malloc(sizeof(int) * nz);
    c->cs = (double *)malloc(sizeof(double) * 2 * nx);
    if (!c->fl || !c->dx || !c->prof || !c->wy || !c->wz || !c->ly || !c->lz || !c->cs) return -2;
    c->sn = c->cs + nx;
    for (int j = 0; j < nx; ++j) { c->cs[j] = cos(2.0 * M_PI * j / nx); c->sn[j] = sin(2.0 * M_PI * j / nx); }
    for (int j = 0; j < ny; ++j) c->ly[j] = fd5(y, ny, j, c->wy + 5 * j);
    for (int j = 0; j < nz; ++j) c->lz[j] = fd5(z, nz, j, c->wz + 5 * j);

    /* mean over x and snapshots at every point of the cross section */
    for (int f = 0; f < 4; ++f)
        for (long p = 0; p < P; ++p) {
            double acc = 0.0;
            for (int s = 0; s < ns; ++s) {
                const double *src = phys + (((long)s * 4 + f) * P + p) * nx;
                for (int x = 0; x < nx; ++x) acc += src[x];
            }
            c->prof[(P_U + f) * P + p] = acc / ((double)ns * nx);
        }
    for (int s = 0; s < ns; ++s)
        for (int f = 0; f < 4; ++f)
            for (long p = 0; p < P; ++p) {
                const double *src = phys + (((long)s * 4 + f) * P + p) * nx;
                double m = c->prof[(P_U + f) * P + p];
                double *dst = FL(c, s, f, p);
                for (int x = 0; x < nx; ++x) dst[x] = src[x] - m;
            }
    /* mean-velocity gradients by the stencils of the y and z grids */
    for (int i = 0; i < 3; ++i)
        for (int iy = 0; iy < ny; ++iy)
            for (int iz = 0; iz < nz; ++iz) {
                double gy = 0.0, gz = 0.0;
                for (int l = 0; l < 5; ++l) {
                    gy += c->wy[5 * iy + l] * c->prof[(P_U + i) * P + (long)(c->ly[iy] + l) * nz + iz];
                    gz += c->wz[5 * iz + l] * c->prof[(P_U + i) * P + (long)iy * nz + c->lz[iz] + l];
                }
                c->prof[(P_G + 2 * i) * P + (long)iy * nz + iz] = gy;
                c->prof[(P_G + 2 * i + 1) * P + (long)iy * nz + iz] = gz;
            }
    /* spectral x derivatives of the fluctuating velocity */
    #pragma omp parallel for schedule(static) collapse(3)
    for (int s = 0; s < ns; ++s)
        for (int i = 0; i < 3; ++i)
            for (long p = 0; p < P; ++p) dft_deriv(FL(c, s, i, p), DXU(c, s, i, p), nx, Lx, c->cs, c->sn);
    /* pseudo-dissipation */
    for (int iy = 0; iy < ny; ++iy)
        for (int iz = 0; iz < nz; ++iz) {
            long p = (long)iy * nz + iz;
            double acc = 0.0;
            for (int s = 0; s < ns; ++s)
                for (int i = 0; i < 3; ++i)
                    for (int x = 0; x < nx; ++x) {
                        double gy = 0.0, gz = 0.0;
                        for (int l = 0; l < 5; ++l) {
                            gy += c->wy[5 * iy + l] * FL(c, s, i, (long)(c->ly[iy] + l) * nz + iz)[x];
                            gz += c->wz[5 * iz + l] * FL(c, s, i, (long)iy * nz + c->lz[iz] + l)[x];
                        }
                        double gx = DXU(c, s, i, p)[x];
                        acc += gx * gx + gy * gy + gz * gz;
                    }
            c->prof[P_EPS * P + p] = nu * acc / ((double)ns * nx);
        }
    return 0;
}

/* direct averages at one ordered pair (p1, p2) and separation m_x:
 * out[0..C_GXA] = A, B_x..z, C_y, C_z, P_y, P_z, Q_ik, R_ik, GxA          */
static void moments(const ctx1h *c, long p1, long p2, int mx, double *out)
{
    int nx = c->nx;
    double acc[C_GXA + 1];
    memset(acc, 0, sizeof(acc));
    for (int s = 0; s < c->ns; ++s) {
        const double *a[4], *b[4], *bx[3];
        for (int f = 0; f < 4; ++f) { a[f] = FL(c, s, f, p1); b[f] = FL(c, s, f, p2); }
        for (int i = 0; i < 3; ++i) bx[i] = DXU(c, s, i, p2);
        for (int x = 0; x < nx; ++x) {
            int xp = (x + mx) % nx;
            double du[3], us[3];
            for (int i = 0; i < 3; ++i) { du[i] = b[i][xp] - a[i][x]; us[i] = 0.5 * (a[i][x] + b[i][xp]); }
            double dp = b[3][xp] - a[3][x];
            double q = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
            acc[C_A] += q;
            acc[C_BX] += q * du[0]; acc[C_BY] += q * du[1]; acc[C_BZ] += q * du[2];
            acc[C_CY] += us[1] * q; acc[C_CZ] += us[2] * q;
            acc[C_PY] += dp * du[1]; acc[C_PZ] += dp * du[2];
            for (int k = 1; k <= 2; ++k)
                for (int i = 0; i < 3; ++i) {
                    acc[C_Q + 3 * (k - 1) + i] += du[i] * du[k];
                    acc[C_R + 3 * (k - 1) + i] += du[i] * us[k];
                }
            acc[C_GXA] += 2.0 * (du[0] * bx[0][xp] + du[1] * bx[1][xp] + du[2] * bx[2][xp]);
        }
    }
    double inv = 1.0 / ((double)c->ns * nx);
    for (int k = 0; k <= C_GXA; ++k) out[k] = acc[k] * inv;
}

/* the terms (all but the residual) from the components at (p1, p2) */
static void assemble(const ctx1h *c, long p1, long p2, const double *cm, double *t)
{
    const double nu = c->nu;
    const long P = c->P;
    const double *pr = c->prof;
    double dU[3], Us[3];
    for (int k = 0; k < 3; ++k) {
        dU[k] = pr[(P_U + k) * P + p2] - pr[(P_U + k) * P + p1];
        Us[k] = 0.5 * (pr[(P_U + k) * P + p1] + pr[(P_U + k) * P + p2]);
    }
    double A = cm[C_A];
    t[T_A] = A;
    t[T_PHIX] = cm[C_BX] + A * dU[0] - 2.0 * nu * cm[C_GXA];
    t[T_PHIY] = cm[C_BY] + A * dU[1] - 2.0 * nu * 0.5 * (cm[C_DY2] - cm[C_DY1]);
    t[T_PHIZ] = cm[C_BZ] + A * dU[2] - 2.0 * nu * 0.5 * (cm[C_DZ2] - cm[C_DZ1]);
    t[T_PSIY] = cm[C_CY] + A * Us[1] + 2.0 * cm[C_PY] - 0.5 * nu * (cm[C_DY1] + cm[C_DY2]);
    t[T_PSIZ] = cm[C_CZ] + A * Us[2] + 2.0 * cm[C_PZ] - 0.5 * nu * (cm[C_DZ1] + cm[C_DZ2]);
    double xi = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int k = 1; k <= 2; ++k) {
            double g1 = pr[(P_G + 2 * i + (k - 1)) * P + p1], g2 = pr[(P_G + 2 * i + (k - 1)) * P + p2];
            xi += -2.0 * cm[C_Q + 3 * (k - 1) + i] * 0.5 * (g1 + g2) - 2.0 * cm[C_R + 3 * (k - 1) + i] * (g2 - g1);
        }
    t[T_XI] = xi - 4.0 * 0.5 * (pr[P_EPS * P + p1] + pr[P_EPS * P + p2]);
}

/* ------------------------------------------------------------------ full run */
int oracle1h_full(const double *phys, int ns, int nx, int ny, int nz, const double *y, const double *z,
                  double Lx, double nu, double *comp, double *terms, double *prof, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    ctx1h c;
    int rc = ctx_init(&c, phys, ns, nx, ny, nz, y, z, Lx, nu);
    if (rc) { ctx_free(&c); return rc; }
    const long P = c.P, sq = P * P;
#define AT(arr, k, a, b) ((arr) + (((long)(k) * sq + (long)(a) * P + (b)) * nx))

    #pragma omp parallel for schedule(dynamic)
    for (long pr = 0; pr < sq; ++pr) {
        double m[C_GXA + 1];
        for (int mx = 0; mx < nx; ++mx) {
            moments(&c, pr / P, pr % P, mx, m);
            for (int k = 0; k <= C_GXA; ++k) comp[((long)k * sq + pr) * nx + mx] = m[k];
        }
    }
    /* Y1, Y2, Z1, Z2 derivatives of A by the stencils */
    #pragma omp parallel for schedule(static)
    for (long pr = 0; pr < sq; ++pr) {
        long p1 = pr / P, p2 = pr % P;
        int iy1 = (int)(p1 / nz), iz1 = (int)(p1 % nz), iy2 = (int)(p2 / nz), iz2 = (int)(p2 % nz);
        for (int mx = 0; mx < nx; ++mx) {
            double d[4] = {0, 0, 0, 0};
            for (int l = 0; l < 5; ++l) {
                d[0] += c.wy[5 * iy1 + l] * AT(comp, C_A, (long)(c.ly[iy1] + l) * nz + iz1, p2)[mx];
                d[1] += c.wy[5 * iy2 + l] * AT(comp, C_A, p1, (long)(c.ly[iy2] + l) * nz + iz2)[mx];
                d[2] += c.wz[5 * iz1 + l] * AT(comp, C_A, (long)iy1 * nz + c.lz[iz1] + l, p2)[mx];
                d[3] += c.wz[5 * iz2 + l] * AT(comp, C_A, p1, (long)iy2 * nz + c.lz[iz2] + l)[mx];
            }
            for (int k = 0; k < 4; ++k) comp[((long)(C_DY1 + k) * sq + pr) * nx + mx] = d[k];
        }
    }
    #pragma omp parallel for schedule(static)
    for (long pr = 0; pr < sq; ++pr) {
        for (int mx = 0; mx < nx; ++mx) {
            double cm[NCOMP], t[NTERM];
            for (int k = 0; k < NCOMP; ++k) cm[k] = comp[((long)k * sq + pr) * nx + mx];
            assemble(&c, pr / P, pr % P, cm, t);
            for (int k = 0; k < T_RES; ++k) terms[((long)k * sq + pr) * nx + mx] = t[k];
        }
    }
    /* residual: spectral r_x derivative, stencils in Y1, Y2, Z1, Z2 */
    #pragma omp parallel for schedule(static)
    for (long pr = 0; pr < sq; ++pr) {
        long p1 = pr / P, p2 = pr % P;
        int iy1 = (int)(p1 / nz), iz1 = (int)(p1 % nz), iy2 = (int)(p2 / nz), iz2 = (int)(p2 % nz);
        double *res = AT(terms, T_RES, p1, p2);
        dft_deriv(AT(terms, T_PHIX, p1, p2), res, nx, Lx, c.cs, c.sn);
        for (int mx = 0; mx < nx; ++mx) {
            double fy1 = 0, fy2 = 0, fz1 = 0, fz2 = 0, sy1 = 0, sy2 = 0, sz1 = 0, sz2 = 0;
            for (int l = 0; l < 5; ++l) {
                long a1 = (long)(c.ly[iy1] + l) * nz + iz1, a2 = (long)(c.ly[iy2] + l) * nz + iz2;
                long b1 = (long)iy1 * nz + c.lz[iz1] + l, b2 = (long)iy2 * nz + c.lz[iz2] + l;
                double w1 = c.wy[5 * iy1 + l], w2 = c.wy[5 * iy2 + l];
                double v1 = c.wz[5 * iz1 + l], v2 = c.wz[5 * iz2 + l];
                fy1 += w1 * AT(terms, T_PHIY, a1, p2)[mx];
                fy2 += w2 * AT(terms, T_PHIY, p1, a2)[mx];
                sy1 += w1 * AT(terms, T_PSIY, a1, p2)[mx];
                sy2 += w2 * AT(terms, T_PSIY, p1, a2)[mx];
                fz1 += v1 * AT(terms, T_PHIZ, b1, p2)[mx];
                fz2 += v2 * AT(terms, T_PHIZ, p1, b2)[mx];
                sz1 += v1 * AT(terms, T_PSIZ, b1, p2)[mx];
                sz2 += v2 * AT(terms, T_PSIZ, p1, b2)[mx];
            }
            res[mx] += 0.5 * (fy2 - fy1) + 0.5 * (fz2 - fz1) + (sy1 + sy2) + (sz1 + sz2)
                       - AT(terms, T_XI, p1, p2)[mx];
        }
    }
#undef AT
    memcpy(prof, c.prof, sizeof(double) * NPROF * P);
    ctx_free(&c);
    return 0;
}

/* --------------------------------------------------------------- spot checks
 * Components and terms (all but the residual) at pts[n][3] = (p1, p2, m_x),
 * any ordered pair; the stencil parts evaluate A directly at the neighbour
 * pairs.  out [n][NCOMP + NTERM - 1].                                      */
int oracle1h_points(const double *phys, int ns, int nx, int ny, int nz, const double *y, const double *z,
                    double Lx, double nu, int npts, const int *pts, double *out, double *prof, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    ctx1h c;
    int rc = ctx_init(&c, phys, ns, nx, ny, nz, y, z, Lx, nu);
    if (rc) { ctx_free(&c); return rc; }
    const long P = c.P;
    for (int q = 0; q < npts; ++q)
        if (pts[3 * q] < 0 || pts[3 * q] >= P || pts[3 * q + 1] < 0 || pts[3 * q + 1] >= P ||
            pts[3 * q + 2] < 0 || pts[3 * q + 2] >= nx) { ctx_free(&c); return -1; }
    const int W = NCOMP + NTERM - 1;
    #pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < npts; ++q) {
        long p1 = pts[3 * q], p2 = pts[3 * q + 1];
        int mx = pts[3 * q + 2];
        int iy1 = (int)(p1 / nz), iz1 = (int)(p1 % nz), iy2 = (int)(p2 / nz), iz2 = (int)(p2 % nz);
        double cm[NCOMP], t[NTERM], m[C_GXA + 1];
        moments(&c, p1, p2, mx, m);
        for (int k = 0; k <= C_GXA; ++k) cm[k] = m[k];
        double d[4] = {0, 0, 0, 0};
        for (int l = 0; l < 5; ++l) {
            moments(&c, (long)(c.ly[iy1] + l) * nz + iz1, p2, mx, m); d[0] += c.wy[5 * iy1 + l] * m[C_A];
            moments(&c, p1, (long)(c.ly[iy2] + l) * nz + iz2, mx, m); d[1] += c.wy[5 * iy2 + l] * m[C_A];
            moments(&c, (long)iy1 * nz + c.lz[iz1] + l, p2, mx, m);   d[2] += c.wz[5 * iz1 + l] * m[C_A];
            moments(&c, p1, (long)iy2 * nz + c.lz[iz2] + l, mx, m);   d[3] += c.wz[5 * iz2 + l] * m[C_A];
        }
        for (int k = 0; k < 4; ++k) cm[C_DY1 + k] = d[k];
        assemble(&c, p1, p2, cm, t);
        for (int k = 0; k < NCOMP; ++k) out[(long)q * W + k] = cm[k];
        for (int k = 0; k < T_RES; ++k) out[(long)q * W + NCOMP + k] = t[k];
    }
    memcpy(prof, c.prof, sizeof(double) * NPROF * P);
    ctx_free(&c);
    return 0;
}
