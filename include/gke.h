/*
 * gke.h -- C ABI of the GB300 Parseval evaluator of the Generalised
 * Kolmogorov Equation (GKE) for plane channel flow.
 *
 * Method: Gatti, Remigi, Chiarini, Cimarelli, Quadrio, "An efficient
 * numerical method for the Generalised Kolmogorov Equation".  The terms of
 * the GKE for the plane channel (Sec. 2, Eq. 2-6) are written as sums of
 * two-point correlations plus one-point moments (Sec. 3.1, Eq. 7); each
 * correlation over the homogeneous directions is the inverse Fourier
 * transform of a product of Fourier coefficients (Parseval, Eq. 8-9); the
 * correlations are averaged over snapshots (Step 2, Sec. 3.2) and the
 * wall-normal derivatives are taken afterwards with a 5-point finite
 * difference stencil in Y1 = Y - r_y/2, Y2 = Y + r_y/2 (Step 3, Eq. 10-11),
 * values across the diagonal Y2 < Y1 coming from r-inversion (Sec. 3.3).
 *
 * Conventions
 *   - Grid: nx x nz points over the periodic box Lx x Lz; ny wall-normal
 *     points y[0..ny) (strictly increasing, walls included, no ghost nodes).
 *   - Input snapshot layout (complex128 = two doubles, re/im interleaved):
 *       fields[nsnap][4][ny][nz][nx/2 + 1]   fields u, v, w, p (mean included)
 *     Coefficients are forward-normalised,
 *       a_hat(y, kz, kx) = 1/(nx nz) sum_{x,z} a(x, y, z) e^{-i (kx x + kz z)},
 *     kz in FFT order (index m -> m for m < nz/2, m - nz above), kx = 0..nx/2:
 *     exactly numpy/torch rfft2(a, norm="forward") over the last two axes.
 *   - Pairs (pair_domain = GKE_DOMAIN_TRIANGLE): the npair = ny (ny + 1) / 2
 *     ordered pairs (i1, i2), i1 <= i2, enumerated row-major (i1 outer);
 *     Y1 = y[i1], Y2 = y[i2]; Y = (Y1 + Y2)/2, r_y = Y2 - Y1
 *     (gke_pair_labels).  Terms at Y2 < Y1 follow from the stored ones by
 *     r-inversion: A, phi, xi are even, Phi_x, Phi_y, Phi_z odd under
 *     (Y1, Y2, r) -> (Y2, Y1, -r).
 *   - Pairs (pair_domain = GKE_DOMAIN_WEDGE, Sec. 3.2 Step 2 and Sec. 3.3):
 *     every snapshot also contributes its mirror image about the centreline,
 *     u(x, 2h - y, z), -v(x, 2h - y, z), w(x, 2h - y, z), p(x, 2h - y, z),
 *     which doubles the statistical sample; the outputs are the pairs of the
 *     half-channel wedge i1 <= i2, i1 + i2 <= ny - 1 (Y1 <= h, Y1 <= Y2 <=
 *     2h - Y1), row-major, npair = sum over i1 of (ny - 2 i1).  The grid must
 *     be symmetric (y[j] + y[ny-1-j] the same for every j).  Terms of the
 *     other pairs follow by r-inversion and by the combined inversion of y
 *     and r, (Y1, Y2, r) -> (2h - Y2, 2h - Y1, -r), under which Phi_x, Phi_z
 *     and phi change sign and A, Phi_y, xi and the residual do not.
 *   - Separations: index (m_z, m_x) in [0, nz) x [0, nx), FFT order,
 *     r_x = m_x Lx / nx, r_z = m_z Lz / nz (periodic).  With undersampling
 *     (Sec. 3.4; desc.under_x / under_z) only the kept indices are stored,
 *     nrz x nrx of them, in increasing order (gke_separation_labels).  Along
 *     each direction, with d = min(m, n - m) the distance from r = 0 in grid
 *     steps and {t1, t2, s1, s2} the option: m is kept when d < t1, or when
 *     t1 <= d < t2 and d is a multiple of s1, or when d >= t2 and d is a
 *     multiple of s2 (0 <= t1 <= t2, s2 >= 1, s1 >= 1 when t1 < t2; else
 *     GKE_ERR_ARG).  All four zero means every m (full resolution); e.g.
 *     {0, 0, 0, 4} keeps every fourth separation.  Thresholded undersampling
 *     selects from the full-resolution result, so the kept values are
 *     exact.  A uniform stride s dividing n in both directions ({0, 0, *, s})
 *     is computed on the coarse grid instead: the spectra are aliased onto
 *     it (exact), the wavenumbers run in chunks, and the per-pair sums shrink
 *     by s_z s_x -- the memory-bounded mode for large grids.  Plans whose
 *     contractions would not fit in memory at once run in the same chunked
 *     mode at stride 1.
 *   - Output terms (double on the FP64 path, float on the FP32 and split paths):
 *       terms[GKE_NTERM][npair][nrz][nrx]     (nrz = nz, nrx = nx at full resolution)
 *     in the order GKE_TERM_* below: <du^2>, Phi_x, Phi_y, Phi_z, phi, xi
 *     and the residual of Eq. 3 (div_r Phi + d phi/dY - xi).
 *   - Profiles (double): profiles[GKE_NPROF][ny], order GKE_PROF_*.
 *
 * Memory: every data pointer may be a device pointer or a host pointer
 * (pageable or pinned); the library detects which.  Host inputs are staged
 * through library-owned device buffers, so the caller may reuse them as soon
 * as the call returns; device inputs must stay valid until the plan's stream
 * reaches the next synchronisation point.  The caller owns every buffer it
 * passes; the plan owns its workspaces and accumulators.
 *
 * Asynchrony: device-pointer calls are asynchronous on the plan's stream,
 * except gke_finalize_terms, which synchronises the stream to read the
 * non-finite-input flag before it returns.
 *
 * Errors: every call returns a gke_status; no call aborts or throws.
 * gke_last_error(plan) (or NULL for gke_plan failures) gives a message.
 */
#ifndef GKE_H
#define GKE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gke_plan_s* gke_plan_t;

typedef enum {
    GKE_OK = 0,
    GKE_ERR_ARG = -1,          /* invalid argument (sizes, NULL pointers)            */
    GKE_ERR_STATE = -2,        /* call out of order (no mean, no samples, finalized) */
    GKE_ERR_OOM = -3,          /* device or host allocation failed                   */
    GKE_ERR_CUDA = -4,         /* a CUDA runtime call failed                         */
    GKE_ERR_NONFINITE = -5,    /* a NaN or Inf was found in the input               */
    GKE_ERR_IO = -6,           /* checkpoint file could not be read or written       */
    GKE_ERR_UNSUPPORTED = -7   /* grid size or option the library does not support   */
} gke_status;

enum { GKE_PREC_F64 = 0,       /* plain FP64 path (DFMA)                              */
       GKE_PREC_BF16X3 = 1,    /* split-BF16 correlator on the tensor cores, FP32 rest */
       GKE_PREC_F32 = 2 };     /* FP32 correlator on the CUDA cores (FFMA), FP32 rest  */

enum { GKE_DOMAIN_TRIANGLE = 0,  /* all pairs i1 <= i2                                  */
       GKE_DOMAIN_WEDGE = 1 };   /* y-inversion mirror sampling, half-channel wedge     */

enum { GKE_TERM_A = 0, GKE_TERM_PHI_X, GKE_TERM_PHI_Y, GKE_TERM_PHI_Z, GKE_TERM_PHI,
       GKE_TERM_XI, GKE_TERM_RESIDUAL, GKE_NTERM };

enum { GKE_PROF_U = 0, GKE_PROF_V, GKE_PROF_W, GKE_PROF_P, GKE_PROF_DUDY, GKE_PROF_EPS, GKE_NPROF };

typedef struct {
    int nx, nz, ny;        /* grid; nx, nz in [8, 1024], 2^a or 3 * 2^a; 5 <= ny <= 1024 */
    double Lx, Lz;         /* box lengths of the homogeneous directions (> 0)            */
    double nu;             /* kinematic viscosity (> 0)                                  */
    const double* y;       /* host pointer, y[ny], strictly increasing; copied            */
    int max_snap;          /* largest nsnap of any accumulate call (sizes workspaces)    */
    int precision;         /* GKE_PREC_*                                                 */
    int pair_domain;       /* GKE_DOMAIN_*                                               */
    int under_x[4];        /* undersampling of r_x {t1, t2, s1, s2}; all 0 = full        */
    int under_z[4];        /* undersampling of r_z, same rule                            */
    unsigned term_mask;    /* terms to compute: bit t = GKE_TERM t; 0 = all (see below)  */
    const char* tune_cache;/* NULL: built-in schedule; else a tuning file (see below)    */
} gke_desc;

/* tune_cache: path of a text file of tuned schedules, one line per device
 * and problem shape.  gke_plan looks the plan's line up; if there is none it
 * times the candidates of each knob on the device (on the plan's workspaces,
 * before any data arrives; results do not depend on the knobs) and appends
 * the fastest: the pair-chunk size of the inverse transforms (scratch W of
 * 48, 96 or 192 MiB per chunk) and the wavenumbers per CTA of the combine
 * kernel (1, 2, 4 on the FP64 path; 2, 4, 8 otherwise).  An unreadable or
 * unwritable file only skips the lookup or the store.  gke_plan_knobs reports
 * what a plan uses.                                                         */

/* term_mask: the plan computes the requested terms and the terms they are
 * derived from -- A for Phi_y and phi (Step-3 FD parts, Eq. 10-11), and A,
 * Phi_y, phi for the residual -- and runs only the contractions those need
 * (A: D; Phi_x: Gx, D; Phi_y: QV, X2; Phi_z: Gz, D; phi: QV, X2, F; xi: E;
 * residual: Gx, Gz, D, E).  Planes of the output outside that set are not
 * written (their contents are unspecified); the planes inside it equal a
 * full run's up to rounding.  Bits above GKE_NTERM: GKE_ERR_ARG.
 * gke_term_set gives the set a mask expands to.  The products pass is the
 * same for every mask (the one-point parts need it).                        */
#define GKE_TERM_BIT(t) (1u << (t))
#define GKE_ALL_TERMS ((1u << GKE_NTERM) - 1u)
unsigned gke_term_set(unsigned term_mask);

/* Create a plan: validates the descriptor, computes the FD weights and
 * twiddles on the host, allocates every workspace on the current device.
 * stream: a cudaStream_t (NULL = legacy default stream).  Nothing is
 * allocated later except the staging buffer of a first host-output finalize. */
gke_status gke_plan(const gke_desc* desc, void* stream, gke_plan_t* out);

/* Step 1 (Sec. 3.2) for databases in velocity-vorticity form: the fields
 * u, v, w, p of nsnap snapshots from the wall-normal velocity v and vorticity
 * eta = du/dz - dw/dx and the plane averages of u and w, for the plan's grid.
 *   v_eta    complex128 [nsnap][2][ny][nz][nx/2+1]: v, eta, forward-normalised
 *            like `fields` (host or device);
 *   mean_uw  float64 [nsnap][2][ny]: the (0, 0) modes of u and w (host or
 *            device);
 *   fields   complex128 [nsnap][4][ny][nz][nx/2+1] out (host or device), the
 *            layout every gke_accumulate_* call reads.
 * u, w (kx^2 + kz^2 > 0): the solution of continuity i kx u + dv/dy + i kz w = 0
 * and eta = i kz u - i kx w; the (0, 0) modes are mean_uw, other modes with
 * kx^2 + kz^2 = 0 are zero.  p: lap p = -d_i d_j (u_i u_j) (rho = 1), the six
 * products of the total velocity formed on the collocation grid, with
 * dp/dy = nu d2v/dy2 at both walls; p(y_0) = 0 fixes the (0, 0) mode.
 * Odd x / z derivatives use the signed wavenumber (0 on the Nyquist lines),
 * second derivatives its true square; d/dy and d2/dy2 are 5-point weights on
 * the nodes of gke_fd_weights.  FP64 throughout, one snapshot at a time; the
 * first call allocates about 13 ny nz (nx/2+1) x 16 bytes of workspace and
 * factors the banded Poisson operators once per plan.  Returns after the
 * last host copy when an argument is in host memory, else asynchronously on
 * the plan's stream.  GKE_ERR_ARG on NULL pointers or nsnap < 1.              */
gke_status gke_velocity_vorticity(gke_plan_t plan, const void* v_eta, const double* mean_uw, int nsnap,
                                  void* fields);

/* Step 1 (Sec. 3.2): add nsnap snapshots to the ensemble mean of u, v, w, p.
 * Only the k = 0 coefficients are read.  Must precede the first
 * gke_accumulate_snapshot; GKE_ERR_STATE afterwards.                         */
gke_status gke_accumulate_mean(gke_plan_t plan, const void* fields, int nsnap);

/* Alternative to gke_accumulate_mean: set the mean profiles directly,
 * mean[4][ny] (u, v, w, p), host or device pointer.                           */
gke_status gke_set_mean(gke_plan_t plan, const double* mean);

/* Step 2 (Sec. 3.2): add nsnap (1 <= nsnap <= max_snap) snapshots to the
 * two-point statistics.  The first call freezes the mean (GKE_ERR_STATE if
 * none was given).  Linear in the snapshots: any split into calls gives the
 * same result up to rounding.  GKE_ERR_STATE after gke_finalize_terms until
 * gke_reset.                                                                 */
gke_status gke_accumulate_snapshot(gke_plan_t plan, const void* fields, int nsnap);

/* Step 3 (Sec. 3.2): write all terms for every pair and separation and,
 * if profiles != NULL, the profiles.  terms holds double on the FP64 path
 * (GKE_PREC_F64) and float otherwise (GKE_PREC_BF16X3, GKE_PREC_F32).  GKE_ERR_STATE without samples;
 * GKE_ERR_NONFINITE if any accumulated input held a NaN or Inf (outputs are
 * then undefined).  May be called again; accumulators are left unchanged.  */
gke_status gke_finalize_terms(gke_plan_t plan, void* terms, double* profiles);

/* One full pass: gke_accumulate_mean + gke_accumulate_snapshot +
 * gke_finalize_terms on a fresh plan state, staging host data once.        */
gke_status gke_compute(gke_plan_t plan, const void* fields, int nsnap, void* terms, double* profiles);

/* gke_compute as one CUDA graph: the first call (and any call with other
 * pointers or nsnap) captures the whole pass -- reset, Step-1 mean frozen on
 * the device, the batch, Step 3 -- from the plan's stream into a graph;
 * later calls replay it.  Device pointers only (else GKE_ERR_ARG); the plan
 * must have been created on a non-default stream (else GKE_ERR_UNSUPPORTED).
 * Results equal gke_compute's; synchronises the stream like
 * gke_finalize_terms.  Not part of the paper: a launch-overhead option.     */
gke_status gke_compute_graph(gke_plan_t plan, const void* fields, int nsnap, void* terms, double* profiles);

/* Host arrays of the pair labels: Y[npair], ry[npair], i1[npair], i2[npair]
 * (any may be NULL).                                                         */
gke_status gke_pair_labels(gke_plan_t plan, double* Y, double* ry, int* i1, int* i2);

/* Sizes: number of pairs, and bytes of the terms array (element size 8 on
 * the FP64 path, 4 otherwise).                                               */
long long gke_npair(gke_plan_t plan);
/* Kept separations: *nrz, *nrx (either may be NULL), and when mz / mx are
 * not NULL the kept indices m_z[nrz], m_x[nrx] (host arrays).              */
gke_status gke_separation_labels(gke_plan_t plan, int* nrz, int* nrx, int* mz, int* mx);
long long gke_terms_bytes(gke_plan_t plan);

/* Schedule of a plan: transform scratch per pair chunk (MiB), wavenumbers
 * per combine CTA, and where they came from (0 built-in, 1 tuning file,
 * 2 measured by this gke_plan).  NULL outputs are skipped.                  */
gke_status gke_plan_knobs(gke_plan_t plan, int* w_chunk_mib, int* comb_kc, int* source);

/* Forget all accumulated statistics and the mean.                            */
gke_status gke_reset(gke_plan_t plan);

/* Save / restore the accumulated state (mean sums, one-point sums, the
 * spectra summed over snapshots, counts) to / from a file; linear, so
 * restored partial sums combine exactly with further calls (the paper's
 * merge of independent jobs, Sec. 3.4).  gke_merge adds a checkpoint's sums
 * to the plan's.  The spectra of a job are taken about the Step-1 mean it
 * froze, so jobs combine exactly only when they share that mean (set it with
 * gke_set_mean, or run gke_accumulate_mean over the same snapshots in every
 * job); gke_merge refuses (GKE_ERR_ARG) a file whose frozen mean differs
 * from the plan's by more than rounding (1e-12 of the largest value).      */
/* File layout (little endian): a header struct { char magic[8] "GKECKPT";
 * int32 version = 5, nx, nz, ny, precision, have_acc, pair_domain, nzt, nxt,
 * term_set (gke_term_set of the plan's mask), acc_kind, reserved; float64
 * mean_count, snap_count, Lx, Lz, nu } (96 bytes), then float64
 * mean_sum[4][ny], float64 stats[7][ny] and, if have_acc, float64 mean[4][ny]
 * (the frozen mean) and the complex128 spectra: acc_kind 0 = per-pair term
 * spectra [npair][GKE_NTERM][nz (nx/2 + 1)], acc_kind 1 = the six plane
 * spectra that split-BF16 plans on the full triangle with ny <= 128 or
 * ny = 129 sum, [6][nz (nx/2 + 1)][npp], npp = npair rounded up to a multiple
 * of 4, acc_kind 2 = the coarse term spectra of the chunked mode (uniform
 * stride, or grids too large for one batch's contractions) for every pair of
 * the triangle, also with the wedge domain, [npair_tri][GKE_NTERM][nzd]
 * [nxd/2 + 1].  Restore and merge need the same
 * grid, domain, term set and acc_kind (else GKE_ERR_ARG).  Files of
 * independent jobs can also be added on the host
 * (paper_1910_06409_gb300/merge.py).                                        */
gke_status gke_checkpoint(gke_plan_t plan, const char* path);
gke_status gke_restore(gke_plan_t plan, const char* path);
gke_status gke_merge(gke_plan_t plan, const char* path);

/* Host utility (no GPU needed): the 5-point first-derivative weights the
 * plan uses at row j of the grid y[ny] (Step 3, Sec. 3.2): w[0..5) on rows
 * l0..l0+4, l0 = clamp(j - 2, 0, ny - 5), exact for polynomials of degree
 * <= 4.  Returns l0, or -1 on bad arguments.                               */
int gke_fd_weights(const double* y, int ny, int j, double* w);

/* Diagnostics.  While timing is on, the plan records CUDA events on its
 * stream around each stage of the path; gke_stage_times synchronises the
 * stream, writes the device milliseconds summed per stage since the last
 * read into ms[GKE_NSTAGE] and clears them.  gke_launch_count is the number
 * of kernels the plan has launched since it was created.                    */
enum { GKE_STAGE_MEAN = 0,       /* Step 1 ensemble mean                          */
       GKE_STAGE_PRODUCTS,       /* fluctuations, in-plane products, one-point sums */
       GKE_STAGE_CORRELATE,      /* per-wavenumber contractions over snapshots    */
       GKE_STAGE_COMBINE,        /* per-pair term spectra, FP64 sum over batches  */
       GKE_STAGE_TERMS,          /* inverse transforms + one-point parts          */
       GKE_STAGE_STENCIL,        /* Step 3 Y1/Y2 finite differences               */
       GKE_NSTAGE };
gke_status gke_set_timing(gke_plan_t plan, int on);
gke_status gke_stage_times(gke_plan_t plan, double* ms);
long long gke_launch_count(gke_plan_t plan);

/* gke_compute without any device allocation, for callers that cannot call
 * cudaMalloc (code running inside a memory pool or allocator it must not
 * re-enter, runtimes that forbid device allocation after start-up).  The
 * paper has no counterpart: this is a deployment variant of the FP64 path.
 * Workspaces come from one file-scope device array of
 * GKE_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits; problems needing more return GKE_ERR_UNSUPPORTED
 * (roughly: nx nz ny^2 <= 2e5 at 2 snapshots, e.g. 16 x 16 x 17; use a plan
 * above that).  nx and nz as for gke_plan (2^a or 3 * 2^a in [8, 1024], else
 * GKE_ERR_UNSUPPORTED); FP64 precision only (desc->precision = GKE_PREC_F64,
 * else GKE_ERR_UNSUPPORTED), the triangle pair domain at full resolution;
 * fields, terms and profiles (may be NULL) must be device pointers (else
 * GKE_ERR_ARG); desc->max_snap is ignored.  The first call on a device finds
 * the array's device address and sets kernel attributes, so make it before
 * any stream capture.  All calls share the array: calls that overlap on the
 * GPU race; each call clears what must start at zero.  Each call uploads its
 * small tables (one copy each) and synchronises `stream` before returning.
 * Status codes only (no message).                                            */
#define GKE_NOALLOC_SCRATCH_BYTES (32u << 20)
gke_status gke_compute_noalloc(const gke_desc* desc, const void* fields, int nsnap, double* terms,
                               double* profiles, void* stream);

/* Message of the last failed call on this plan (plan == NULL: last gke_plan
 * failure of the calling thread).  Valid until the next call on the plan.  */
const char* gke_last_error(gke_plan_t plan);

/* Free every resource of the plan (synchronises its stream).  NULL is a no-op. */
void gke_destroy(gke_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* GKE_H */
