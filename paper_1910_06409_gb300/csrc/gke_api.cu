// gke_api.cu -- the plan object and the C ABI declared in include/gke.h.
//
// Host-side work only: validation, FD weights (Fornberg's recursion on the
// non-uniform wall-normal grid), FFT twiddles, the pair table, workspace
// allocation and the launch sequence of Steps 1-3.  Every arithmetic step of
// the path itself runs in the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gke.h"
#include "gke_common.cuh"
#include "gke_kernels.h"
#include "gke_split.h"

using namespace gke;

struct gke_plan_s {
    gke_desc d;
    std::vector<double> y;
    cudaStream_t st = nullptr;
    int nxh = 0, Nk = 0;
    long long npair = 0;
    // device workspaces
    zd *Xop = nullptr, *G = nullptr, *H = nullptr, *acc_sq = nullptr, *acc_D = nullptr, *W = nullptr;
    zd *tw_x = nullptr, *tw_z = nullptr, *stage_in = nullptr;
    double *mean_sum = nullptr, *mean = nullptr, *stats = nullptr, *prof = nullptr, *fdw = nullptr;
    double *stage_terms = nullptr, *stage_prof = nullptr, *part = nullptr;
    size_t part_count = 0;
    int *fdl0 = nullptr, *pair_i = nullptr, *nonfinite = nullptr;
    SplitWork split;
    long long pair_chunk = 0;
    // diagnostics
    bool timing = false;
    long long launches = 0;
    struct Mark { int stage; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> spare;
    // host state
    double mean_count = 0.0, snap_count = 0.0;
    bool mean_frozen = false, have_acc = false, finalized = false;
    std::string err;
};

static thread_local std::string g_plan_err;

#define CUDA_TRY(plan, call)                                                                \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            (plan)->err = std::string(#call) + ": " + cudaGetErrorString(e_);               \
            return e_ == cudaErrorMemoryAllocation ? GKE_ERR_OOM : GKE_ERR_CUDA;            \
        }                                                                                   \
    } while (0)

static gke_status fail(gke_plan_t p, gke_status s, const std::string& m) { p->err = m; return s; }

static cudaEvent_t take_event(gke_plan_t p)
{
    if (!p->spare.empty()) { cudaEvent_t e = p->spare.back(); p->spare.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// stage timing: begin / end record events on the plan's stream when enabled
struct StageScope {
    gke_plan_t p; int stage; cudaEvent_t a = nullptr;
    StageScope(gke_plan_t p_, int s) : p(p_), stage(s) {
        if (p->timing) { a = take_event(p); cudaEventRecord(a, p->st); }
    }
    ~StageScope() {
        if (p->timing && a) {
            cudaEvent_t b = take_event(p);
            cudaEventRecord(b, p->st);
            p->marks.push_back({stage, a, b});
        }
    }
};

// ------------------------------------------------------------- host helpers
// First-derivative weights at z0 on the nodes x[0..n) by Fornberg's recursion
// (B. Fornberg, Math. Comp. 51 (1988) 699-706), written for derivative
// orders 0 and 1 only.
static void fornberg_d1(const double* x, int n, double z0, double* w)
{
    std::vector<double> c0(n, 0.0), c1(n, 0.0);
    double prod_prev = 1.0;
    double dz_prev = x[0] - z0;
    c0[0] = 1.0;
    for (int i = 1; i < n; ++i) {
        double prod = 1.0;
        double dz_i = x[i] - z0;
        for (int j = 0; j < i; ++j) {
            double dx = x[i] - x[j];
            prod *= dx;
            if (j == i - 1) {
                // new node i from node i-1's weights
                c1[i] = prod_prev * (c0[i - 1] - dz_prev * c1[i - 1]) / prod;
                c0[i] = -prod_prev * dz_prev * c0[i - 1] / prod;
            }
            c1[j] = (dz_i * c1[j] - c0[j]) / dx;
            c0[j] = dz_i * c0[j] / dx;
        }
        prod_prev = prod;
        dz_prev = dz_i;
    }
    for (int i = 0; i < n; ++i) w[i] = c1[i];
}

static const int EPS_KCHUNK = 64;

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int smem_limit()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// tile parameters of the transform kernels for a grid (bounded by shared memory)
struct Tiles { int cw_ci, rz_rp, cw_cf, yb_cf, cw_tc, rz_tr; };
static Tiles pick_tiles(int nx, int nz)
{
    Tiles t;
    const int lim = 96 * 1024;   // keep two CTAs per SM possible
    t.cw_ci = 8; while (t.cw_ci > 1 && t.cw_ci * nz * 16 > lim) t.cw_ci /= 2;
    t.rz_rp = 4; while (t.rz_rp > 1 && t.rz_rp * 6 * nx * 16 > lim) t.rz_rp /= 2;
    t.cw_cf = 4; t.yb_cf = 4; while (t.cw_cf * t.yb_cf > 1 && t.cw_cf * t.yb_cf * nz * 16 > lim) {
        if (t.yb_cf > 1) t.yb_cf /= 2; else t.cw_cf /= 2; }
    t.cw_tc = 4; while (t.cw_tc > 1 && NTERM * t.cw_tc * nz * 16 > lim) t.cw_tc /= 2;
    t.rz_tr = 4; while (t.rz_tr > 1 && t.rz_tr * 4 * nx * 16 > lim) t.rz_tr /= 2;
    return t;
}

static cudaError_t set_smem_attrs()
{
    int lim = smem_limit();
    cudaError_t e = cudaSuccess;
    const void* ks[] = {(const void*)k_col_inverse, (const void*)k_row_products, (const void*)k_col_forward,
                        (const void*)k_terms_colpass, (const void*)k_terms_rowpass};
    for (const void* k : ks) {
        cudaFuncAttributes fa;
        cudaError_t r = cudaFuncGetAttributes(&fa, k);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - (int)fa.sharedSizeBytes);
        if (r != cudaSuccess) e = r;
    }
    return e;
}

template <typename T> static cudaError_t dalloc(T** p, size_t count)
{
    return cudaMalloc((void**)p, count * sizeof(T));
}

// ------------------------------------------------------------------- plan
extern "C" gke_status gke_plan(const gke_desc* desc, void* stream, gke_plan_t* out)
{
    if (!out) { g_plan_err = "out is NULL"; return GKE_ERR_ARG; }
    *out = nullptr;
    if (!desc || !desc->y) { g_plan_err = "desc or desc->y is NULL"; return GKE_ERR_ARG; }
    const gke_desc& d = *desc;
    if (d.nx < 8 || d.nz < 8 || d.nx > 1024 || d.nz > 1024 || d.ny < 5 || d.ny > 1024 || d.max_snap < 1) {
        g_plan_err = "grid sizes out of range (8 <= nx, nz <= 1024, 5 <= ny <= 1024, max_snap >= 1)";
        return GKE_ERR_ARG;
    }
    if (!(d.Lx > 0) || !(d.Lz > 0) || !(d.nu > 0)) { g_plan_err = "Lx, Lz, nu must be > 0"; return GKE_ERR_ARG; }
    if (!is_pow2(d.nx) || !is_pow2(d.nz)) {
        g_plan_err = "nx and nz must be powers of two in this build";
        return GKE_ERR_UNSUPPORTED;
    }
    if (d.precision != GKE_PREC_F64 && d.precision != GKE_PREC_BF16X3) {
        g_plan_err = "unknown precision";
        return GKE_ERR_ARG;
    }
    for (int j = 1; j < d.ny; ++j)
        if (!(d.y[j] > d.y[j - 1])) { g_plan_err = "y must be strictly increasing"; return GKE_ERR_ARG; }

    gke_plan_t p = new (std::nothrow) gke_plan_s;
    if (!p) { g_plan_err = "host allocation failed"; return GKE_ERR_OOM; }
    p->d = d;
    p->y.assign(d.y, d.y + d.ny);
    p->d.y = p->y.data();
    p->st = (cudaStream_t)stream;
    p->nxh = d.nx / 2 + 1;
    p->Nk = d.nz * p->nxh;
    p->npair = (long long)d.ny * (d.ny + 1) / 2;
    const int ny = d.ny, ns = d.max_snap, Nk = p->Nk;
    const size_t plane = (size_t)d.nz * p->nxh;

    auto bail = [&](gke_status s, const std::string& m) { g_plan_err = m; gke_destroy(p); return s; };
    cudaError_t e;
#define ALLOC(ptr, n)                                                                          \
    do {                                                                                       \
        e = dalloc(&(ptr), (size_t)(n));                                                       \
        if (e != cudaSuccess) return bail(GKE_ERR_OOM, std::string("cudaMalloc " #ptr ": ") +  \
                                                           cudaGetErrorString(e));             \
    } while (0)
    ALLOC(p->Xop, (size_t)NFIELD * Nk * ns * ny);
    ALLOC(p->G, (size_t)4 * ny * plane);
    ALLOC(p->H, (size_t)7 * ny * plane);
    ALLOC(p->acc_sq, (size_t)NJSQ * ny * ny * Nk);
    ALLOC(p->acc_D, (size_t)p->npair * Nk);
    p->pair_chunk = std::max<long long>(1, std::min<long long>(p->npair, (2LL << 30) / ((long long)NTERM * Nk * 16)));
    ALLOC(p->W, (size_t)p->pair_chunk * NTERM * Nk);
    ALLOC(p->tw_x, d.nx / 2);
    ALLOC(p->tw_z, d.nz / 2);
    ALLOC(p->mean_sum, 4 * ny);
    ALLOC(p->mean, 4 * ny);
    ALLOC(p->stats, NSTAT * ny);
    ALLOC(p->prof, NPR * ny);
    ALLOC(p->fdw, 5 * ny);
    ALLOC(p->fdl0, ny);
    ALLOC(p->pair_i, 2 * p->npair);
    ALLOC(p->nonfinite, 1);
    {
        const Tiles tl = pick_tiles(d.nx, d.nz);
        size_t a1 = (size_t)6 * ny * ((d.nz + tl.rz_rp - 1) / tl.rz_rp);
        size_t a2 = (size_t)ny * ((Nk + EPS_KCHUNK - 1) / EPS_KCHUNK);
        p->part_count = std::max(a1, a2);
        ALLOC(p->part, p->part_count);
    }
    if (d.precision == GKE_PREC_BF16X3) {
        gke_status s = split_alloc(p->split, ny, ns, Nk);
        if (s != GKE_OK) return bail(s, "split workspace allocation failed");
    }
#undef ALLOC
    // host tables
    std::vector<zd> twx(d.nx / 2), twz(d.nz / 2);
    for (int m = 0; m < d.nx / 2; ++m) { twx[m].x = std::cos(2.0 * M_PI * m / d.nx); twx[m].y = -std::sin(2.0 * M_PI * m / d.nx); }
    for (int m = 0; m < d.nz / 2; ++m) { twz[m].x = std::cos(2.0 * M_PI * m / d.nz); twz[m].y = -std::sin(2.0 * M_PI * m / d.nz); }
    std::vector<double> w(5 * ny);
    std::vector<int> l0(ny);
    for (int j = 0; j < ny; ++j) {
        int a = std::min(std::max(j - 2, 0), ny - 5);
        l0[j] = a;
        fornberg_d1(p->y.data() + a, 5, p->y[j], w.data() + 5 * j);
    }
    std::vector<int> pi(2 * p->npair);
    long long q = 0;
    for (int i1 = 0; i1 < ny; ++i1)
        for (int i2 = i1; i2 < ny; ++i2) { pi[2 * q] = i1; pi[2 * q + 1] = i2; ++q; }
    cudaStream_t st = p->st;
    if ((e = cudaMemcpyAsync(p->tw_x, twx.data(), twx.size() * sizeof(zd), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(p->tw_z, twz.data(), twz.size() * sizeof(zd), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(p->fdw, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(p->fdl0, l0.data(), l0.size() * sizeof(int), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(p->pair_i, pi.data(), pi.size() * sizeof(int), cudaMemcpyHostToDevice, st)) ||
        (e = cudaStreamSynchronize(st)))
        return bail(GKE_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    if ((e = set_smem_attrs()) != cudaSuccess) return bail(GKE_ERR_CUDA, std::string("smem attr: ") + cudaGetErrorString(e));
    upload_jobs(st);
    if (d.precision == GKE_PREC_BF16X3) {
        if ((e = split_setup(st)) != cudaSuccess) return bail(GKE_ERR_CUDA, std::string("split setup: ") + cudaGetErrorString(e));
    }
    gke_status rs = gke_reset(p);
    if (rs != GKE_OK) return bail(rs, p->err);
    *out = p;
    return GKE_OK;
}

extern "C" gke_status gke_reset(gke_plan_t p)
{
    if (!p) return GKE_ERR_ARG;
    CUDA_TRY(p, cudaMemsetAsync(p->mean_sum, 0, 4 * p->d.ny * sizeof(double), p->st));
    CUDA_TRY(p, cudaMemsetAsync(p->stats, 0, NSTAT * p->d.ny * sizeof(double), p->st));
    CUDA_TRY(p, cudaMemsetAsync(p->nonfinite, 0, sizeof(int), p->st));
    p->mean_count = 0.0;
    p->snap_count = 0.0;
    p->mean_frozen = p->have_acc = p->finalized = false;
    return GKE_OK;
}

extern "C" void gke_destroy(gke_plan_t p)
{
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st); else cudaDeviceSynchronize();
    void* ptrs[] = {p->Xop, p->G, p->H, p->acc_sq, p->acc_D, p->W, p->tw_x, p->tw_z, p->stage_in,
                    p->mean_sum, p->mean, p->stats, p->prof, p->fdw, p->stage_terms, p->stage_prof,
                    p->fdl0, p->pair_i, p->nonfinite, p->part};
    for (void* q : ptrs) if (q) cudaFree(q);
    split_free(p->split);
    for (auto& m : p->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
    for (auto e : p->spare) cudaEventDestroy(e);
    delete p;
}

extern "C" int gke_fd_weights(const double* y, int ny, int j, double* w)
{
    if (!y || !w || ny < 5 || j < 0 || j >= ny) return -1;
    int a = std::min(std::max(j - 2, 0), ny - 5);
    fornberg_d1(y + a, 5, y[j], w);
    return a;
}

extern "C" gke_status gke_set_timing(gke_plan_t p, int on)
{
    if (!p) return GKE_ERR_ARG;
    p->timing = on != 0;
    return GKE_OK;
}

extern "C" gke_status gke_stage_times(gke_plan_t p, double* ms)
{
    if (!p || !ms) return p ? fail(p, GKE_ERR_ARG, "ms is NULL") : GKE_ERR_ARG;
    CUDA_TRY(p, cudaStreamSynchronize(p->st));
    for (int s = 0; s < GKE_NSTAGE; ++s) ms[s] = 0.0;
    for (auto& m : p->marks) {
        float t = 0.f;
        CUDA_TRY(p, cudaEventElapsedTime(&t, m.a, m.b));
        ms[m.stage] += t;
        p->spare.push_back(m.a);
        p->spare.push_back(m.b);
    }
    p->marks.clear();
    return GKE_OK;
}

extern "C" long long gke_launch_count(gke_plan_t p) { return p ? p->launches : -1; }

extern "C" const char* gke_last_error(gke_plan_t p) { return p ? p->err.c_str() : g_plan_err.c_str(); }
extern "C" long long gke_npair(gke_plan_t p) { return p ? p->npair : -1; }
extern "C" long long gke_terms_bytes(gke_plan_t p)
{
    return p ? (long long)NTERM * p->npair * p->d.nx * p->d.nz * (long long)sizeof(double) : -1;
}

extern "C" gke_status gke_pair_labels(gke_plan_t p, double* Y, double* ry, int* i1, int* i2)
{
    if (!p) return GKE_ERR_ARG;
    long long q = 0;
    for (int a = 0; a < p->d.ny; ++a)
        for (int b = a; b < p->d.ny; ++b, ++q) {
            if (Y) Y[q] = 0.5 * (p->y[a] + p->y[b]);
            if (ry) ry[q] = p->y[b] - p->y[a];
            if (i1) i1[q] = a;
            if (i2) i2[q] = b;
        }
    return GKE_OK;
}

// device pointer to the snapshot data: stages host data into stage_in
static gke_status device_fields(gke_plan_t p, const void* fields, int nsnap, const zd** out)
{
    if (is_device_ptr(fields)) { *out = (const zd*)fields; return GKE_OK; }
    const size_t bytes = (size_t)nsnap * 4 * p->d.ny * p->Nk * sizeof(zd);
    if (!p->stage_in) CUDA_TRY(p, dalloc(&p->stage_in, (size_t)p->d.max_snap * 4 * p->d.ny * p->Nk));
    CUDA_TRY(p, cudaMemcpyAsync(p->stage_in, fields, bytes, cudaMemcpyHostToDevice, p->st));
    *out = p->stage_in;
    return GKE_OK;
}

static gke_status mean_impl(gke_plan_t p, const zd* f, int nsnap)
{
    const int ny = p->d.ny;
    {
        StageScope sc(p, GKE_STAGE_MEAN);
        k_mean_accum<<<(4 * ny + 127) / 128, 128, 0, p->st>>>(f, nsnap, ny, (long long)p->Nk, p->mean_sum);
        p->launches += 1;
    }
    CUDA_TRY(p, cudaGetLastError());
    p->mean_count += nsnap;
    return GKE_OK;
}

extern "C" gke_status gke_accumulate_mean(gke_plan_t p, const void* fields, int nsnap)
{
    if (!p || !fields) return p ? fail(p, GKE_ERR_ARG, "fields is NULL") : GKE_ERR_ARG;
    if (nsnap < 1 || nsnap > p->d.max_snap) return fail(p, GKE_ERR_ARG, "nsnap out of range [1, max_snap]");
    if (p->mean_frozen) return fail(p, GKE_ERR_STATE, "mean is frozen: snapshots were already accumulated");
    const zd* f;
    gke_status s = device_fields(p, fields, nsnap, &f);
    if (s != GKE_OK) return s;
    return mean_impl(p, f, nsnap);
}

extern "C" gke_status gke_set_mean(gke_plan_t p, const double* mean)
{
    if (!p || !mean) return p ? fail(p, GKE_ERR_ARG, "mean is NULL") : GKE_ERR_ARG;
    if (p->mean_frozen) return fail(p, GKE_ERR_STATE, "mean is frozen: snapshots were already accumulated");
    CUDA_TRY(p, cudaMemcpyAsync(p->mean_sum, mean, 4 * p->d.ny * sizeof(double), cudaMemcpyDefault, p->st));
    p->mean_count = 1.0;
    return GKE_OK;
}

static gke_status snapshot_impl(gke_plan_t p, const zd* f, int ns)
{
    const gke_desc& d = p->d;
    const int ny = d.ny, Nk = p->Nk, nxh = p->nxh;
    cudaStream_t st = p->st;
    if (!p->mean_frozen) {
        // mean = mean_sum / mean_count, computed once (host round trip of 4 ny doubles)
        std::vector<double> m(4 * ny);
        CUDA_TRY(p, cudaMemcpyAsync(m.data(), p->mean_sum, m.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(p, cudaStreamSynchronize(st));
        for (double& v : m) v /= p->mean_count;
        CUDA_TRY(p, cudaMemcpyAsync(p->mean, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        CUDA_TRY(p, cudaStreamSynchronize(st));
        p->mean_frozen = true;
    }
    const Tiles t = pick_tiles(d.nx, d.nz);
    dim3 b32(32, 8);
    StageScope* sc_prod = new StageScope(p, GKE_STAGE_PRODUCTS);
    k_load_linear<<<dim3((Nk + 31) / 32, (ny + 31) / 32, ns * 4), b32, 0, st>>>(f, ns, ny, Nk, p->mean, p->Xop,
                                                                              p->nonfinite);
    for (int s = 0; s < ns; ++s) {
        const zd* fs = f + (size_t)s * 4 * ny * Nk;
        k_col_inverse<<<dim3((nxh + t.cw_ci - 1) / t.cw_ci, ny, 4), 256, t.cw_ci * d.nz * sizeof(zd), st>>>(
            fs, ny, d.nz, nxh, t.cw_ci, p->mean, p->tw_z, p->G);
        const int nrb = (d.nz + t.rz_rp - 1) / t.rz_rp;
        k_row_products<<<dim3(nrb, ny), 256, t.rz_rp * 6 * d.nx * sizeof(zd), st>>>(
            p->G, ny, d.nz, d.nx, t.rz_rp, p->tw_x, p->H, p->part);
        k_reduce_partials<<<(6 * ny + 127) / 128, 128, 0, st>>>(p->part, 6 * ny, nrb, p->stats);
        p->launches += 3;
        k_col_forward<<<dim3((nxh + t.cw_cf - 1) / t.cw_cf, (ny + t.yb_cf - 1) / t.yb_cf, 7), 256,
                        t.cw_cf * t.yb_cf * d.nz * sizeof(zd), st>>>(p->H, ny, d.nz, nxh, t.cw_cf, t.yb_cf, s, ns,
                                                                     p->tw_z, p->Xop);
        p->launches += 1;
    }
    const int neb = (Nk + EPS_KCHUNK - 1) / EPS_KCHUNK;
    k_eps<<<neb, 128, 0, st>>>(p->Xop, ns, ny, d.nz, nxh, d.nx, d.Lx, d.Lz, p->fdw, p->fdl0, EPS_KCHUNK, p->part);
    k_reduce_partials<<<(ny + 127) / 128, 128, 0, st>>>(p->part, ny, neb, p->stats + S_EPS * ny);
    p->launches += 3;
    delete sc_prod;
    StageScope sc_corr(p, GKE_STAGE_CORRELATE);
    if (d.precision == GKE_PREC_F64) {
        k_correlate_f64<<<dim3(Nk, NJSQ + 1), 256, 0, st>>>(p->Xop, ns, ny, Nk, p->have_acc ? 1 : 0, p->acc_sq,
                                                             p->acc_D);
        p->launches += 1;
    } else {
        int nl = 0;
        gke_status s = split_correlate(p->split, p->Xop, ns, ny, Nk, p->have_acc ? 1 : 0, p->acc_sq, p->acc_D, st,
                                       p->err, &nl);
        p->launches += nl;
        if (s != GKE_OK) return s;
    }
    CUDA_TRY(p, cudaGetLastError());
    p->snap_count += ns;
    p->have_acc = true;
    return GKE_OK;
}

extern "C" gke_status gke_accumulate_snapshot(gke_plan_t p, const void* fields, int nsnap)
{
    if (!p || !fields) return p ? fail(p, GKE_ERR_ARG, "fields is NULL") : GKE_ERR_ARG;
    if (nsnap < 1 || nsnap > p->d.max_snap) return fail(p, GKE_ERR_ARG, "nsnap out of range [1, max_snap]");
    if (p->finalized) return fail(p, GKE_ERR_STATE, "plan was finalized: call gke_reset first");
    if (!p->mean_frozen && p->mean_count <= 0) return fail(p, GKE_ERR_STATE, "no mean: call gke_accumulate_mean or gke_set_mean first");
    const zd* f;
    gke_status s = device_fields(p, fields, nsnap, &f);
    if (s != GKE_OK) return s;
    return snapshot_impl(p, f, nsnap);
}

static gke_status finalize_impl(gke_plan_t p, double* terms_dev)
{
    const gke_desc& d = p->d;
    const int ny = d.ny, nxh = p->nxh;
    cudaStream_t st = p->st;
    const Tiles t = pick_tiles(d.nx, d.nz);
    StageScope* sc_terms = new StageScope(p, GKE_STAGE_TERMS);
    k_profiles<<<(ny + 127) / 128, 128, 0, st>>>(p->mean_sum, p->mean_count, p->stats, p->snap_count,
                                                  (long long)d.nx * d.nz, d.nu, p->fdw, p->fdl0, ny, p->prof);
    const double inv_count = 1.0 / p->snap_count;
    for (long long p0 = 0; p0 < p->npair; p0 += p->pair_chunk) {
        long long np = std::min(p->pair_chunk, p->npair - p0);
        k_terms_colpass<<<dim3((nxh + t.cw_tc - 1) / t.cw_tc, (unsigned)np), 256, NTERM * t.cw_tc * d.nz * sizeof(zd),
                          st>>>(p->acc_sq, p->acc_D, p->pair_i, p0, ny, d.nz, d.nx, t.cw_tc, d.Lx, d.Lz, d.nu,
                                inv_count, p->prof, p->tw_z, p->W);
        k_terms_rowpass<<<dim3((d.nz + t.rz_tr - 1) / t.rz_tr, (unsigned)np), 256, t.rz_tr * 4 * d.nx * sizeof(zd),
                          st>>>(p->W, p->pair_i, p0, p->npair, ny, d.nz, d.nx, t.rz_tr, p->prof, p->tw_x, terms_dev);
        p->launches += 2;
    }
    p->launches += 1;
    delete sc_terms;
    StageScope sc_st(p, GKE_STAGE_STENCIL);
    const long long N = (long long)d.nx * d.nz;
    dim3 gs((unsigned)((N + 255) / 256), (unsigned)p->npair);
    k_stencil_A<<<gs, 256, 0, st>>>(terms_dev, p->npair, p->pair_i, ny, d.nz, d.nx, d.nu, p->fdw, p->fdl0);
    k_stencil_res<<<gs, 256, 0, st>>>(terms_dev, p->npair, p->pair_i, ny, d.nz, d.nx, p->fdw, p->fdl0);
    p->launches += 2;
    CUDA_TRY(p, cudaGetLastError());
    return GKE_OK;
}

// user-visible profiles [GKE_NPROF][ny] are the first GKE_NPROF rows of prof
static_assert((int)PR_U == (int)GKE_PROF_U && (int)PR_V == (int)GKE_PROF_V && (int)PR_W == (int)GKE_PROF_W &&
              (int)PR_P == (int)GKE_PROF_P && (int)PR_DU == (int)GKE_PROF_DUDY && (int)PR_EPS == (int)GKE_PROF_EPS,
              "profile order");

extern "C" gke_status gke_finalize_terms(gke_plan_t p, double* terms, double* profiles)
{
    if (!p || !terms) return p ? fail(p, GKE_ERR_ARG, "terms is NULL") : GKE_ERR_ARG;
    if (!p->have_acc || p->snap_count <= 0) return fail(p, GKE_ERR_STATE, "no snapshots accumulated");
    const bool dev_out = is_device_ptr(terms);
    const size_t tbytes = (size_t)gke_terms_bytes(p);
    double* tdev = terms;
    if (!dev_out) {
        if (!p->stage_terms) CUDA_TRY(p, dalloc(&p->stage_terms, tbytes / sizeof(double)));
        tdev = p->stage_terms;
    }
    gke_status s = finalize_impl(p, tdev);
    if (s != GKE_OK) return s;
    if (!dev_out) CUDA_TRY(p, cudaMemcpyAsync(terms, tdev, tbytes, cudaMemcpyDeviceToHost, p->st));
    if (profiles)
        CUDA_TRY(p, cudaMemcpyAsync(profiles, p->prof, GKE_NPROF * p->d.ny * sizeof(double), cudaMemcpyDefault, p->st));
    int bad = 0;
    CUDA_TRY(p, cudaMemcpyAsync(&bad, p->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(p, cudaStreamSynchronize(p->st));
    p->finalized = true;
    if (p->d.precision == GKE_PREC_BF16X3) {
        gke_status ss = split_check(p->split, p->st, p->err);
        if (ss != GKE_OK) return ss;
    }
    if (bad) return fail(p, GKE_ERR_NONFINITE, "non-finite value in the accumulated input");
    return GKE_OK;
}

extern "C" gke_status gke_compute(gke_plan_t p, const void* fields, int nsnap, double* terms, double* profiles)
{
    if (!p || !fields || !terms) return p ? fail(p, GKE_ERR_ARG, "NULL argument") : GKE_ERR_ARG;
    if (nsnap < 1 || nsnap > p->d.max_snap) return fail(p, GKE_ERR_ARG, "nsnap out of range [1, max_snap]");
    gke_status s = gke_reset(p);
    if (s != GKE_OK) return s;
    const zd* f;
    if ((s = device_fields(p, fields, nsnap, &f)) != GKE_OK) return s;
    if ((s = mean_impl(p, f, nsnap)) != GKE_OK) return s;
    if ((s = snapshot_impl(p, f, nsnap)) != GKE_OK) return s;
    return gke_finalize_terms(p, terms, profiles);
}

// ------------------------------------------------------- checkpoint files
struct CkptHeader {
    char magic[8];
    int version, nx, nz, ny, precision, have_acc;
    double mean_count, snap_count, Lx, Lz, nu;
};

static gke_status ckpt_io(gke_plan_t p, const char* path, int mode)   // 0 save, 1 restore, 2 merge
{
    if (!p || !path) return p ? fail(p, GKE_ERR_ARG, "path is NULL") : GKE_ERR_ARG;
    const int ny = p->d.ny;
    const size_t n_mean = 4 * ny, n_stat = (size_t)NSTAT * ny;
    const size_t n_sq = (size_t)NJSQ * ny * ny * p->Nk, n_D = (size_t)p->npair * p->Nk;
    CUDA_TRY(p, cudaStreamSynchronize(p->st));
    if (mode == 0) {
        FILE* fp = fopen(path, "wb");
        if (!fp) return fail(p, GKE_ERR_IO, std::string("cannot open for writing: ") + path);
        CkptHeader h{};
        memcpy(h.magic, "GKECKPT", 8);
        h.version = 1; h.nx = p->d.nx; h.nz = p->d.nz; h.ny = ny; h.precision = p->d.precision;
        h.have_acc = p->have_acc; h.mean_count = p->mean_count; h.snap_count = p->snap_count;
        h.Lx = p->d.Lx; h.Lz = p->d.Lz; h.nu = p->d.nu;
        bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
        std::vector<char> buf;
        auto put = [&](const void* dptr, size_t bytes) {
            buf.resize(bytes);
            if (cudaMemcpy(buf.data(), dptr, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
            return fwrite(buf.data(), 1, bytes, fp) == bytes;
        };
        ok = ok && put(p->mean_sum, n_mean * 8) && put(p->stats, n_stat * 8);
        if (p->have_acc) ok = ok && put(p->acc_sq, n_sq * 16) && put(p->acc_D, n_D * 16);
        ok = (fclose(fp) == 0) && ok;
        return ok ? GKE_OK : fail(p, GKE_ERR_IO, std::string("write failed: ") + path);
    }
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(p, GKE_ERR_IO, std::string("cannot open for reading: ") + path);
    CkptHeader h{};
    if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, "GKECKPT", 8) != 0 || h.version != 1) {
        fclose(fp);
        return fail(p, GKE_ERR_IO, "not a GKE checkpoint");
    }
    if (h.nx != p->d.nx || h.nz != p->d.nz || h.ny != ny || h.Lx != p->d.Lx || h.Lz != p->d.Lz || h.nu != p->d.nu) {
        fclose(fp);
        return fail(p, GKE_ERR_ARG, "checkpoint grid does not match the plan");
    }
    if (mode == 2 && p->mean_frozen && h.mean_count > 0 && !p->have_acc) {
        fclose(fp);
        return fail(p, GKE_ERR_STATE, "cannot merge into a plan with a frozen mean and no samples");
    }
    std::vector<char> buf;
    bool ok = true;
    auto get = [&](void* dptr, size_t bytes, bool add_double, bool add_complex) {
        if (!ok) return;
        buf.resize(bytes);
        if (fread(buf.data(), 1, bytes, fp) != bytes) { ok = false; return; }
        if (!add_double && !add_complex) {
            ok = cudaMemcpy(dptr, buf.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
            return;
        }
        std::vector<char> cur(bytes);
        if (cudaMemcpy(cur.data(), dptr, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) { ok = false; return; }
        double* a = (double*)cur.data();
        const double* b = (const double*)buf.data();
        for (size_t i = 0; i < bytes / 8; ++i) a[i] += b[i];
        ok = cudaMemcpy(dptr, cur.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    const bool add = (mode == 2);
    get(p->mean_sum, n_mean * 8, add, false);
    get(p->stats, n_stat * 8, add, false);
    if (h.have_acc) {
        const bool add_acc = add && p->have_acc;
        get(p->acc_sq, n_sq * 16, false, add_acc);
        get(p->acc_D, n_D * 16, false, add_acc);
    }
    fclose(fp);
    if (!ok) return fail(p, GKE_ERR_IO, std::string("read failed or truncated: ") + path);
    if (add) {
        p->mean_count += h.mean_count;
        p->snap_count += h.snap_count;
        p->have_acc = p->have_acc || h.have_acc;
    } else {
        p->mean_count = h.mean_count;
        p->snap_count = h.snap_count;
        p->have_acc = h.have_acc;
    }
    p->mean_frozen = false;
    if (p->have_acc) {
        // the mean used by accumulated snapshots is the stored one: refreeze it
        std::vector<double> m(4 * ny);
        CUDA_TRY(p, cudaMemcpy(m.data(), p->mean_sum, m.size() * 8, cudaMemcpyDeviceToHost));
        for (double& v : m) v /= p->mean_count;
        CUDA_TRY(p, cudaMemcpy(p->mean, m.data(), m.size() * 8, cudaMemcpyHostToDevice));
        p->mean_frozen = true;
    }
    p->finalized = false;
    return GKE_OK;
}

extern "C" gke_status gke_checkpoint(gke_plan_t p, const char* path) { return ckpt_io(p, path, 0); }
extern "C" gke_status gke_restore(gke_plan_t p, const char* path) { return ckpt_io(p, path, 1); }
extern "C" gke_status gke_merge(gke_plan_t p, const char* path) { return ckpt_io(p, path, 2); }
