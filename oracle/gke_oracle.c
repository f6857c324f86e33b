/*
 * gke_oracle.c -- CPU oracle for the GKE terms of plane channel flow.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path never does.  It shares no code, header, table or helper with the CUDA
 * path.
 *
 * What it computes (Gatti et al., "An efficient numerical method for the
 * Generalised Kolmogorov Equation"):
 *
 *   Every GKE term straight from its definition in Sec. 2, as an average of
 *   products of velocity / pressure increments over snapshots and over the
 *   homogeneous directions x, z -- the direct O(N_t N^2) evaluation the paper
 *   contrasts its method with (Sec. 1).  No correlation expansion (Eq. 7)
 *   and no Parseval step (Eq. 8-9) is used, so agreement with the Parseval
 *   path pins both.
 *
 *   For planes Y1 = y[i1], Y2 = y[i2] and a separation (m_x, m_z) on the
 *   periodic grid, x' = x + r with r = (m_x Lx/nx, m_z Lz/nz):
 *     delta u_i = u_i(x', Y2) - u_i(x, Y1),  delta p likewise,
 *     v*        = (v(x, Y1) + v(x', Y2)) / 2
 *   averaged over x, z and snapshots:
 *     A    = <du_i du_i>                (Eq. 1, the structure function)
 *     B_j  = <du_i du_i du_j>           (turbulent part of Eq. 4)
 *     C    = <v* du_i du_i>             (turbulent part of Eq. 5)
 *     P    = <dp dv>                    (pressure part of Eq. 5, rho = 1)
 *     Q    = <du dv>,  R = <du v*>      (Eq. 6)
 *     GxA  = dA/dr_x = <2 du_i (d_x u_i)(x', Y2)>   (exact: only u_i(x') moves with r)
 *     GzA  = dA/dr_z likewise
 *   wall-normal derivatives by a 5-point finite-difference stencil (Step 3):
 *     dA/dr_y = (d_Y2 - d_Y1) A / 2,   dA/dY = (d_Y1 + d_Y2) A       (Eq. 10-11)
 *   and the terms
 *     Phi_x = B_x + A dU - 2 nu GxA                     (Eq. 4, dU = U(Y2) - U(Y1))
 *     Phi_y = B_y - 2 nu dA/dr_y
 *     Phi_z = B_z - 2 nu GzA
 *     phi   = C + 2 P - (nu/2) dA/dY                    (Eq. 5)
 *     xi    = -2 Q (U')* - 2 R d(U') - 4 eps*           (Eq. 6)
 *     res   = dPhi_x/dr_x + dPhi_y/dr_y + dPhi_z/dr_z + dphi/dY - xi   (Eq. 3)
 *   where * is the mean of the values at Y1 and Y2, eps = nu <d_j u_i d_j u_i>
 *   (pseudo-dissipation, Sec. 2), homogeneous derivatives are spectral (naive
 *   DFT, Nyquist wavenumber taken as zero) and r_y / Y derivatives use the same
 *   FD stencil (Sec. 4.3).  Fluctuations are taken about the ensemble mean
 *   (mean over x, z and snapshots, Step 1).
 *
 * Readings where the paper is silent:
 *   - averages are means over grid points and snapshots (the paper writes
 *     unnormalised integrals);
 *   - the FD stencil is the unique 5-point first-derivative formula exact for
 *     polynomials of degree <= 4 on nodes j-2..j+2 of the (non-uniform) grid,
 *     the window shifted to 0..4 / n-5..n-1 at the two rows nearest a wall;
 *     here its weights come from solving the 5x5 moment (Vandermonde) system;
 *   - all ordered pairs (i1, i2) are computed directly (no symmetry is used),
 *     so the FD windows never need values from across the diagonal.
 *
 * Layouts (C order):
 *   phys  double [ns][4][ny][nz][nx]   fields u, v, w, p including the mean
 *   comp  double [NCOMP][ny][ny][nz][nx]  (full square of ordered pairs)
 *   terms double [NTERM][ny][ny][nz][nx]
 *   prof  double [NPROF][ny]
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { C_A = 0, C_BX, C_BY, C_BZ, C_C, C_P, C_Q, C_R, C_GX, C_GZ, C_DY1, C_DY2, NCOMP };
enum { T_A = 0, T_PHIX, T_PHIY, T_PHIZ, T_PHI, T_XI, T_RES, NTERM };
enum { P_U = 0, P_V, P_W, P_P, P_DU, P_EPS, NPROF };

int oracle_ncomp(void) { return NCOMP; }
int oracle_nterm(void) { return NTERM; }
int oracle_nprof(void) { return NPROF; }

/* ---------------------------------------------------------------- FD weights
 * Solve sum_l w_l t_l^p = [p == 1], p = 0..4, with t_l = y[l0+l] - y[j],
 * after scaling t by h = max |t_l| for conditioning.  Gaussian elimination
 * with partial pivoting on the 5x5 system.  Returns the window start l0.   */
int oracle_fd_weights(const double *y, int ny, int j, double *w)
{
    int l0 = j - 2;
    if (l0 < 0) l0 = 0;
    if (l0 > ny - 5) l0 = ny - 5;
    double t[5], h = 0.0;
    for (int l = 0; l < 5; ++l) {
        t[l] = y[l0 + l] - y[j];
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

/* --------------------------------------------------- naive DFT derivative
 * d/dx of a real periodic sequence f[0..n) with period L: forward DFT
 * F(m) = (1/n) sum_x f(x) e^{-2 pi i m x / n}, multiply by i k_m with
 * k_m = 2 pi m'/L, m' the signed index (m for m < n/2, m - n for m > n/2,
 * 0 at m = n/2), and transform back.  stride = distance between elements.  */
static void naive_deriv(const double *f, double *df, int n, int stride, double L,
                        const double *cs, const double *sn)
{
    double *re = (double *)malloc(sizeof(double) * n * 2);
    double *im = re + n;
    for (int m = 0; m < n; ++m) {
        double ar = 0.0, ai = 0.0;
        for (int x = 0; x < n; ++x) {
            int ph = (int)(((long)m * x) % n);
            ar += f[(long)x * stride] * cs[ph];
            ai -= f[(long)x * stride] * sn[ph];
        }
        ar /= n; ai /= n;
        int ms = (m < n / 2) ? m : m - n;
        if (2 * m == n) ms = 0;
        double k = 2.0 * M_PI * ms / L;
        /* (ar + i ai) * (i k) = -k ai + i k ar */
        re[m] = -k * ai;
        im[m] = k * ar;
    }
    for (int x = 0; x < n; ++x) {
        double acc = 0.0;
        for (int m = 0; m < n; ++m) {
            int ph = (int)(((long)m * x) % n);
            acc += re[m] * cs[ph] - im[m] * sn[ph];
        }
        df[(long)x * stride] = acc;
    }
    free(re);
}

static void trig_table(int n, double *cs, double *sn)
{
    for (int p = 0; p < n; ++p) {
        cs[p] = cos(2.0 * M_PI * p / n);
        sn[p] = sin(2.0 * M_PI * p / n);
    }
}

/* d/dx and d/dz of one plane [nz][nx] */
static void plane_derivs(const double *f, double *fx, double *fz, int nx, int nz,
                         double Lx, double Lz)
{
    double *cx = (double *)malloc(sizeof(double) * 2 * (nx + nz));
    double *sx = cx + nx, *cz = sx + nx, *sz = cz + nz;
    trig_table(nx, cx, sx);
    trig_table(nz, cz, sz);
    for (int z = 0; z < nz; ++z) naive_deriv(f + (long)z * nx, fx + (long)z * nx, nx, 1, Lx, cx, sx);
    for (int x = 0; x < nx; ++x) naive_deriv(f + x, fz + x, nz, nx, Lz, cz, sz);
    free(cx);
}

/* ----------------------------------------------------------- shared state */
typedef struct {
    int ns, nx, nz, ny;
    double Lx, Lz, nu;
    const double *y;
    long N;                 /* nx * nz */
    double *fl;             /* fluctuations [ns][4][ny][N] */
    double **dx, **dz;      /* [ns][3][ny] -> plane [N], allocated only where needed */
    char *have_d;           /* [ny] derivative planes computed */
    double prof[NPROF * 1024];
    double *fdw;            /* [ny][5] */
    int *fdl0;              /* [ny] */
} ctx_t;

#define FL(c, s, f, j) ((c)->fl + ((((long)(s) * 4 + (f)) * (c)->ny + (j)) * (c)->N))
#define DX(c, s, i, j) ((c)->dx[((long)(s) * 3 + (i)) * (c)->ny + (j)])
#define DZ(c, s, i, j) ((c)->dz[((long)(s) * 3 + (i)) * (c)->ny + (j)])

static int ctx_init(ctx_t *c, const double *phys, int ns, int nx, int nz, int ny,
                    const double *y, double Lx, double Lz, double nu)
{
    memset(c, 0, sizeof(*c));
    if (ns < 1 || nx < 2 || nz < 2 || ny < 5 || ny > 1024) return -1;
    c->ns = ns; c->nx = nx; c->nz = nz; c->ny = ny;
    c->Lx = Lx; c->Lz = Lz; c->nu = nu; c->y = y;
    c->N = (long)nx * nz;
    long plane_count = (long)ns * 4 * ny;
    c->fl = (double *)malloc(sizeof(double) * plane_count * c->N);
    c->dx = (double **)calloc((size_t)ns * 3 * ny, sizeof(double *));
    c->dz = (double **)calloc((size_t)ns * 3 * ny, sizeof(double *));
    c->have_d = (char *)calloc(ny, 1);
    c->fdw = (double *)malloc(sizeof(double) * 5 * ny);
    c->fdl0 = (int *)malloc(sizeof(int) * ny);
    if (!c->fl || !c->dx || !c->dz || !c->have_d || !c->fdw || !c->fdl0) return -2;
    memset(c->prof, 0, sizeof(c->prof));

    /* Step 1: ensemble mean of every field, then fluctuations */
    for (int f = 0; f < 4; ++f)
        for (int j = 0; j < ny; ++j) {
            double acc = 0.0;
            for (int s = 0; s < ns; ++s) {
                const double *src = phys + (((long)s * 4 + f) * ny + j) * c->N;
                for (long q = 0; q < c->N; ++q) acc += src[q];
            }
            c->prof[f * ny + j] = acc / ((double)ns * c->N);
        }
    for (int s = 0; s < ns; ++s)
        for (int f = 0; f < 4; ++f)
            for (int j = 0; j < ny; ++j) {
                const double *src = phys + (((long)s * 4 + f) * ny + j) * c->N;
                double *dst = FL(c, s, f, j);
                double m = c->prof[f * ny + j];
                for (long q = 0; q < c->N; ++q) dst[q] = src[q] - m;
            }
    for (int j = 0; j < ny; ++j) c->fdl0[j] = oracle_fd_weights(y, ny, j, c->fdw + 5 * j);
    /* dU/dy by the FD stencil */
    for (int j = 0; j < ny; ++j) {
        double acc = 0.0;
        for (int l = 0; l < 5; ++l) acc += c->fdw[5 * j + l] * c->prof[P_U * ny + c->fdl0[j] + l];
        c->prof[P_DU * ny + j] = acc;
    }
    return 0;
}

static void ctx_free(ctx_t *c)
{
    if (c->dx)
        for (long k = 0; k < (long)c->ns * 3 * c->ny; ++k) { free(c->dx[k]); free(c->dz[k]); }
    free(c->fl); free(c->dx); free(c->dz); free(c->have_d); free(c->fdw); free(c->fdl0);
}

/* spectral x/z derivatives of u_i on the planes flagged in `need` */
static void ctx_derivs(ctx_t *c, const char *need)
{
    int ny = c->ny;
    for (int j = 0; j < ny; ++j)
        for (int s = 0; s < c->ns; ++s)
            for (int i = 0; i < 3; ++i)
                if (need[j] && !c->have_d[j]) {
                    DX(c, s, i, j) = (double *)malloc(sizeof(double) * c->N);
                    DZ(c, s, i, j) = (double *)malloc(sizeof(double) * c->N);
                }
    #pragma omp parallel for schedule(dynamic) collapse(3)
    for (int j = 0; j < ny; ++j)
        for (int s = 0; s < c->ns; ++s)
            for (int i = 0; i < 3; ++i) {
                if (!need[j] || c->have_d[j]) continue;
                plane_derivs(FL(c, s, i, j), DX(c, s, i, j), DZ(c, s, i, j), c->nx, c->nz, c->Lx, c->Lz);
            }
    for (int j = 0; j < ny; ++j) if (need[j]) c->have_d[j] = 1;
}

/* pseudo-dissipation eps(j) = nu <d_x u_i^2 + d_y u_i^2 + d_z u_i^2>; needs derivs at j */
static double ctx_eps(const ctx_t *c, int j)
{
    double acc = 0.0;
    int l0 = c->fdl0[j];
    const double *w = c->fdw + 5 * j;
    for (int s = 0; s < c->ns; ++s)
        for (int i = 0; i < 3; ++i) {
            const double *ax = DX(c, s, i, j), *az = DZ(c, s, i, j);
            for (long q = 0; q < c->N; ++q) {
                double dy = 0.0;
                for (int l = 0; l < 5; ++l) dy += w[l] * FL(c, s, i, l0 + l)[q];
                acc += ax[q] * ax[q] + az[q] * az[q] + dy * dy;
            }
        }
    return c->nu * acc / ((double)c->ns * c->N);
}

/* Direct average of the increment moments at one ordered pair / separation.
 * out[0..9] = A, Bx, By, Bz, C, P, Q, R, GxA, GzA.  with_g: also GxA, GzA. */
static void point_moments(const ctx_t *c, int i1, int i2, int mz, int mx, double *out, int with_g)
{
    int nx = c->nx, nz = c->nz;
    double A = 0, Bx = 0, By = 0, Bz = 0, C = 0, P = 0, Q = 0, R = 0, Gx = 0, Gz = 0;
    for (int s = 0; s < c->ns; ++s) {
        const double *u1 = FL(c, s, 0, i1), *v1 = FL(c, s, 1, i1), *w1 = FL(c, s, 2, i1), *p1 = FL(c, s, 3, i1);
        const double *u2 = FL(c, s, 0, i2), *v2 = FL(c, s, 1, i2), *w2 = FL(c, s, 2, i2), *p2 = FL(c, s, 3, i2);
        const double *ux2 = DX(c, s, 0, i2), *vx2 = DX(c, s, 1, i2), *wx2 = DX(c, s, 2, i2);
        const double *uz2 = DZ(c, s, 0, i2), *vz2 = DZ(c, s, 1, i2), *wz2 = DZ(c, s, 2, i2);
        for (int z = 0; z < nz; ++z) {
            int zp = (z + mz) % nz;
            for (int x = 0; x < nx; ++x) {
                int xp = (x + mx) % nx;
                long a = (long)z * nx + x, b = (long)zp * nx + xp;
                double du = u2[b] - u1[a], dv = v2[b] - v1[a], dw = w2[b] - w1[a];
                double dp = p2[b] - p1[a];
                double vs = 0.5 * (v1[a] + v2[b]);
                double q = du * du + dv * dv + dw * dw;
                A += q;
                Bx += q * du; By += q * dv; Bz += q * dw;
                C += vs * q;
                P += dp * dv;
                Q += du * dv;
                R += du * vs;
                if (with_g) {
                    Gx += 2.0 * (du * ux2[b] + dv * vx2[b] + dw * wx2[b]);
                    Gz += 2.0 * (du * uz2[b] + dv * vz2[b] + dw * wz2[b]);
                }
            }
        }
    }
    double inv = 1.0 / ((double)c->ns * c->N);
    out[0] = A * inv; out[1] = Bx * inv; out[2] = By * inv; out[3] = Bz * inv;
    out[4] = C * inv; out[5] = P * inv; out[6] = Q * inv; out[7] = R * inv;
    out[8] = Gx * inv; out[9] = Gz * inv;
}

/* assemble the terms (all but the residual) from the components at one point */
static void assemble(const ctx_t *c, int i1, int i2, const double *cm, double e1, double e2, double *t)
{
    const double nu = c->nu;
    int ny = c->ny;
    double U1 = c->prof[P_U * ny + i1], U2 = c->prof[P_U * ny + i2];
    double dU1 = c->prof[P_DU * ny + i1], dU2 = c->prof[P_DU * ny + i2];
    double dAry = 0.5 * (cm[C_DY2] - cm[C_DY1]);
    double dAY = cm[C_DY1] + cm[C_DY2];
    t[T_A] = cm[C_A];
    t[T_PHIX] = cm[C_BX] + cm[C_A] * (U2 - U1) - 2.0 * nu * cm[C_GX];
    t[T_PHIY] = cm[C_BY] - 2.0 * nu * dAry;
    t[T_PHIZ] = cm[C_BZ] - 2.0 * nu * cm[C_GZ];
    t[T_PHI] = cm[C_C] + 2.0 * cm[C_P] - 0.5 * nu * dAY;
    t[T_XI] = -2.0 * cm[C_Q] * 0.5 * (dU1 + dU2) - 2.0 * cm[C_R] * (dU2 - dU1) - 4.0 * 0.5 * (e1 + e2);
}

/* --------------------------------------------------------------- full run */
int oracle_full(const double *phys, int ns, int nx, int nz, int ny, const double *y,
                double Lx, double Lz, double nu, double *comp, double *terms, double *prof,
                int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    ctx_t c;
    int rc = ctx_init(&c, phys, ns, nx, nz, ny, y, Lx, Lz, nu);
    if (rc) { ctx_free(&c); return rc; }
    long N = c.N;
    long sq = (long)ny * ny;
    char *need = (char *)malloc(ny);
    memset(need, 1, ny);
    ctx_derivs(&c, need);
    free(need);
    double *eps = c.prof + P_EPS * ny;
    for (int j = 0; j < ny; ++j) eps[j] = ctx_eps(&c, j);

    /* increment moments on every ordered pair and separation */
    #pragma omp parallel for schedule(dynamic)
    for (long pr = 0; pr < sq; ++pr) {
        int i1 = (int)(pr / ny), i2 = (int)(pr % ny);
        double m[10];
        for (int mz = 0; mz < nz; ++mz)
            for (int mx = 0; mx < nx; ++mx) {
                point_moments(&c, i1, i2, mz, mx, m, 1);
                long o = pr * N + (long)mz * nx + mx;
                for (int k = 0; k < 10; ++k) comp[(long)k * sq * N + o] = m[k];
            }
    }
    /* Y1 / Y2 derivatives of A by the FD stencil (Step 3) */
    #pragma omp parallel for schedule(static)
    for (long pr = 0; pr < sq; ++pr) {
        int i1 = (int)(pr / ny), i2 = (int)(pr % ny);
        const double *w1 = c.fdw + 5 * i1, *w2 = c.fdw + 5 * i2;
        int a1 = c.fdl0[i1], a2 = c.fdl0[i2];
        for (long q = 0; q < N; ++q) {
            double d1 = 0.0, d2 = 0.0;
            for (int l = 0; l < 5; ++l) {
                d1 += w1[l] * comp[((long)C_A * sq + (long)(a1 + l) * ny + i2) * N + q];
                d2 += w2[l] * comp[((long)C_A * sq + (long)i1 * ny + (a2 + l)) * N + q];
            }
            comp[((long)C_DY1 * sq + pr) * N + q] = d1;
            comp[((long)C_DY2 * sq + pr) * N + q] = d2;
        }
    }
    /* terms */
    #pragma omp parallel for schedule(static)
    for (long pr = 0; pr < sq; ++pr) {
        int i1 = (int)(pr / ny), i2 = (int)(pr % ny);
        for (long q = 0; q < N; ++q) {
            double cm[NCOMP], t[NTERM];
            for (int k = 0; k < NCOMP; ++k) cm[k] = comp[((long)k * sq + pr) * N + q];
            assemble(&c, i1, i2, cm, eps[i1], eps[i2], t);
            for (int k = 0; k < T_RES; ++k) terms[((long)k * sq + pr) * N + q] = t[k];
        }
    }
    /* residual of Eq. 3: spectral r_x / r_z derivatives, FD r_y / Y derivatives */
    {
        double *cx = (double *)malloc(sizeof(double) * 2 * (nx + nz));
        double *sx = cx + nx, *cz = sx + nx, *sz = cz + nz;
        trig_table(nx, cx, sx);
        trig_table(nz, cz, sz);
        #pragma omp parallel for schedule(static)
        for (long pr = 0; pr < sq; ++pr) {
            int i1 = (int)(pr / ny), i2 = (int)(pr % ny);
            double *res = terms + ((long)T_RES * sq + pr) * N;
            const double *fx = terms + ((long)T_PHIX * sq + pr) * N;
            const double *fz = terms + ((long)T_PHIZ * sq + pr) * N;
            double *tmp = (double *)malloc(sizeof(double) * N);
            for (int z = 0; z < nz; ++z) naive_deriv(fx + (long)z * nx, res + (long)z * nx, nx, 1, Lx, cx, sx);
            for (int x = 0; x < nx; ++x) naive_deriv(fz + x, tmp + x, nz, nx, Lz, cz, sz);
            const double *w1 = c.fdw + 5 * i1, *w2 = c.fdw + 5 * i2;
            int a1 = c.fdl0[i1], a2 = c.fdl0[i2];
            for (long q = 0; q < N; ++q) {
                double y1y = 0.0, y2y = 0.0, y1p = 0.0, y2p = 0.0;
                for (int l = 0; l < 5; ++l) {
                    long o1 = (long)(a1 + l) * ny + i2, o2 = (long)i1 * ny + (a2 + l);
                    y1y += w1[l] * terms[((long)T_PHIY * sq + o1) * N + q];
                    y2y += w2[l] * terms[((long)T_PHIY * sq + o2) * N + q];
                    y1p += w1[l] * terms[((long)T_PHI * sq + o1) * N + q];
                    y2p += w2[l] * terms[((long)T_PHI * sq + o2) * N + q];
                }
                res[q] += tmp[q] + 0.5 * (y2y - y1y) + (y1p + y2p) - terms[((long)T_XI * sq + pr) * N + q];
            }
            free(tmp);
        }
        free(cx);
    }
    for (int k = 0; k < NPROF; ++k)
        for (int j = 0; j < ny; ++j) prof[k * ny + j] = c.prof[k * ny + j];
    ctx_free(&c);
    return 0;
}

/* ------------------------------------------------------------ spot checks
 * Terms (all but the residual) and components at selected points
 * pts[n][4] = (i1, i2, m_z, m_x), any ordered pair.  For the FD parts the
 * structure function is evaluated directly at the stencil's neighbour pairs.
 * out [n][NCOMP + NTERM - 1].  Cost per point ~ 11 ns nx nz.               */
int oracle_points(const double *phys, int ns, int nx, int nz, int ny, const double *y,
                  double Lx, double Lz, double nu, int npts, const int *pts, double *out,
                  double *prof, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    ctx_t c;
    int rc = ctx_init(&c, phys, ns, nx, nz, ny, y, Lx, Lz, nu);
    if (rc) { ctx_free(&c); return rc; }
    char *need = (char *)calloc(ny, 1);
    for (int p = 0; p < npts; ++p) {
        int i1 = pts[4 * p], i2 = pts[4 * p + 1];
        if (i1 < 0 || i1 >= ny || i2 < 0 || i2 >= ny || pts[4 * p + 2] < 0 || pts[4 * p + 2] >= nz ||
            pts[4 * p + 3] < 0 || pts[4 * p + 3] >= nx) { free(need); ctx_free(&c); return -1; }
        need[i1] = need[i2] = 1;
    }
    ctx_derivs(&c, need);
    double *eps = c.prof + P_EPS * ny;
    for (int j = 0; j < ny; ++j) eps[j] = need[j] ? ctx_eps(&c, j) : NAN;
    const int W = NCOMP + NTERM - 1;
    #pragma omp parallel for schedule(dynamic)
    for (int p = 0; p < npts; ++p) {
        int i1 = pts[4 * p], i2 = pts[4 * p + 1], mz = pts[4 * p + 2], mx = pts[4 * p + 3];
        double cm[NCOMP], t[NTERM], m[10];
        point_moments(&c, i1, i2, mz, mx, m, 1);
        for (int k = 0; k < 10; ++k) cm[k] = m[k];
        const double *w1 = c.fdw + 5 * i1, *w2 = c.fdw + 5 * i2;
        int a1 = c.fdl0[i1], a2 = c.fdl0[i2];
        double d1 = 0.0, d2 = 0.0;
        for (int l = 0; l < 5; ++l) {
            point_moments(&c, a1 + l, i2, mz, mx, m, 0);
            d1 += w1[l] * m[0];
            point_moments(&c, i1, a2 + l, mz, mx, m, 0);
            d2 += w2[l] * m[0];
        }
        cm[C_DY1] = d1; cm[C_DY2] = d2;
        assemble(&c, i1, i2, cm, eps[i1], eps[i2], t);
        for (int k = 0; k < NCOMP; ++k) out[(long)p * W + k] = cm[k];
        for (int k = 0; k < T_RES; ++k) out[(long)p * W + NCOMP + k] = t[k];
    }
    for (int k = 0; k < NPROF; ++k)
        for (int j = 0; j < ny; ++j) prof[k * ny + j] = c.prof[k * ny + j];
    free(need);
    ctx_free(&c);
    return 0;
}
