// gke_noalloc.cu -- gke_compute_noalloc: the FP64 path for small grids
// without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool or
// an allocator it must not re-enter, or a host runtime that forbids device
// allocation after start-up.  For them this entry point takes its workspaces
// from one file-scope device array of GKE_NOALLOC_SCRATCH_BYTES (32 MiB)
// instead of a plan.  Every GPU that loads the library holds that array
// until the process exits.  The array's host-side name is only a stand-in:
// the device address comes from cudaGetSymbolAddress, once per device, on
// the device's first call (which also sets the kernels' shared-memory limits
// and constants), so that first call should come before any stream capture.
//
// Every call uses the same array: calls that overlap on the GPU (on two
// streams, or from two threads) race, and each call re-initialises the parts
// that must start at zero.  Nothing here is allocated: no cudaMalloc,
// cudaFree or allocating library routine is called, and the small host
// tables (twiddles, finite-difference weights) live in fixed-size stack
// buffers; the pair table is built on the device.  Each call uploads the
// tables with one copy per table and synchronises the stream before it
// returns.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "../../include/gke.h"
#include "gke_common.cuh"
#include "gke_kernels.h"

using namespace gke;

static __device__ __align__(256) unsigned char g_noalloc_scratch[GKE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
unsigned char* g_scratch_dev[MAX_DEVICES] = {nullptr};   // device address of the array, per device
// status only: this entry point keeps no message (its callers read the code),
// so the texts below are documentation and nothing is formatted
gke_status fail(gke_status s, const char*) { return s; }

// one-time set-up on the current device: array address, kernel attributes, constants
gke_status setup_device(int dev, cudaStream_t st)
{
    if (g_scratch_dev[dev]) return GKE_OK;
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(GKE_ERR_CUDA, "cudaGetSymbolAddress failed");
    int lim = 0;
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((e = products_set_attrs(lim)) != cudaSuccess || (e = terms_set_attrs(lim)) != cudaSuccess ||
        (e = combine_set_attrs()) != cudaSuccess)
        return fail(GKE_ERR_CUDA, "kernel attributes");
    upload_jobs(st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(GKE_ERR_CUDA, "set-up");
    g_scratch_dev[dev] = (unsigned char*)ptr;
    return GKE_OK;
}

// bump carve of the scratch array (256-byte aligned pieces)
struct Carve {
    unsigned char* base;
    size_t off = 0, cap;
    template <typename T> T* take(size_t count)
    {
        size_t o = (off + 255) & ~(size_t)255;
        off = o + count * sizeof(T);
        return (T*)(base + o);
    }
    bool ok() const { return off <= cap; }
};

__global__ void k_div(const double* __restrict__ s, double c, int n, double* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = s[i] / c;
}

// pair_i[2 q], pair_i[2 q + 1] = (i1, i2) of the row-major triangle pair q
__global__ void k_pair_table(int ny, int* __restrict__ pair_i)
{
    const int i1 = blockIdx.x;
    const long long q0 = pair_index(i1, i1, ny);
    for (int i2 = i1 + threadIdx.x; i2 < ny; i2 += blockDim.x) {
        pair_i[2 * (q0 + i2 - i1)] = i1;
        pair_i[2 * (q0 + i2 - i1) + 1] = i2;
    }
}

constexpr int MAX_N = 1024;        // largest nx, nz, ny (the plan's limits)

bool is_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" gke_status gke_compute_noalloc(const gke_desc* desc, const void* fields, int nsnap, double* terms,
                                          double* profiles, void* stream)
{
    if (!desc || !desc->y || !fields || !terms) return fail(GKE_ERR_ARG, "NULL argument");
    const gke_desc& d = *desc;
    if (d.precision != GKE_PREC_F64) return fail(GKE_ERR_UNSUPPORTED, "gke_compute_noalloc runs the FP64 path only");
    if (d.pair_domain != GKE_DOMAIN_TRIANGLE)
        return fail(GKE_ERR_UNSUPPORTED, "gke_compute_noalloc computes the triangle pair domain only");
    for (int i = 0; i < 4; ++i)
        if (d.under_x[i] || d.under_z[i])
            return fail(GKE_ERR_UNSUPPORTED, "gke_compute_noalloc writes full-resolution separations only");
    if (d.nx < 8 || d.nz < 8 || d.nx > MAX_N || d.nz > MAX_N || d.ny < 5 || d.ny > MAX_N || nsnap < 1)
        return fail(GKE_ERR_ARG, "sizes out of range (8 <= nx, nz <= 1024, 5 <= ny <= 1024, nsnap >= 1)");
    if (!fft_len_ok(d.nx) || !fft_len_ok(d.nz))
        return fail(GKE_ERR_UNSUPPORTED, "nx and nz must be 2^a or 3 * 2^a (transform lengths of the library)");
    if (!(d.Lx > 0) || !(d.Lz > 0) || !(d.nu > 0)) return fail(GKE_ERR_ARG, "Lx, Lz, nu must be > 0");
    if (d.term_mask & ~GKE_ALL_TERMS) return fail(GKE_ERR_ARG, "term_mask has bits above GKE_NTERM");
    const unsigned tset = term_set(d.term_mask);
    for (int j = 1; j < d.ny; ++j)
        if (!(d.y[j] > d.y[j - 1])) return fail(GKE_ERR_ARG, "y must be strictly increasing");
    if (!is_device(fields) || !is_device(terms) || (profiles && !is_device(profiles)))
        return fail(GKE_ERR_ARG, "gke_compute_noalloc takes device pointers only");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return fail(GKE_ERR_CUDA, "no device");
    gke_status s = setup_device(dev, st);
    if (s != GKE_OK) return s;

    const int nx = d.nx, nz = d.nz, ny = d.ny, nxh = nx / 2 + 1, Nk = nz * nxh, ns = nsnap;
    const long long npair = (long long)ny * (ny + 1) / 2;
    // transform tiles and partial sums as the plan path sizes them (complex128)
    const Tiles tl = pick_tiles(nx, nz, sizeof(zd));

    Carve c{g_scratch_dev[dev], 0, (size_t)GKE_NOALLOC_SCRATCH_BYTES};
    zd* Xop = c.take<zd>((size_t)NFIELD * Nk * ns * ny);
    zd* G = c.take<zd>((size_t)4 * ny * Nk);
    zd* H = c.take<zd>((size_t)7 * ny * Nk);
    zd* raw = c.take<zd>((size_t)NJOB * ((ny + 7) / 8) * ((ny + 7) / 8) * 64 * Nk);
    zd* comb = c.take<zd>((size_t)npair * NTERM * Nk);
    zd* W = c.take<zd>((size_t)npair * NTERM * Nk);
    zd* twx = c.take<zd>(nx);
    zd* twz = c.take<zd>(nz);
    double* mean_sum = c.take<double>(4 * ny);
    double* mean = c.take<double>(4 * ny);
    double* stats = c.take<double>(NSTAT * ny);
    double* prof = c.take<double>(NPR * ny);
    double* fdw = c.take<double>(5 * ny);
    int* fdl0 = c.take<int>(ny);
    int* pair_i = c.take<int>(2 * npair);
    int* nonfinite = c.take<int>(1);
    double* part = c.take<double>(part_count(nz, ny, Nk, tl));
    if (!c.ok())
        return fail(GKE_ERR_UNSUPPORTED, "workspace larger than GKE_NOALLOC_SCRATCH_BYTES: use a plan (gke_plan)");

    // host tables (libm twiddles, FD weights) in fixed-size stack buffers, one
    // copy per table and one synchronisation before the buffers go out of
    // scope; the pair list is built on the device
    cudaError_t e;
#define TRY(call) do { if ((e = (call)) != cudaSuccess) return fail(GKE_ERR_CUDA, #call); } while (0)
    zd h_twx[MAX_N], h_twz[MAX_N];
    double h_fdw[5 * MAX_N];
    int h_fdl0[MAX_N];
    for (int m = 0; m < nx; ++m) { h_twx[m].x = std::cos(2.0 * M_PI * m / nx); h_twx[m].y = -std::sin(2.0 * M_PI * m / nx); }
    for (int m = 0; m < nz; ++m) { h_twz[m].x = std::cos(2.0 * M_PI * m / nz); h_twz[m].y = -std::sin(2.0 * M_PI * m / nz); }
    for (int j = 0; j < ny; ++j) h_fdl0[j] = gke_fd_weights(d.y, ny, j, h_fdw + 5 * j);
    TRY(cudaMemcpyAsync(twx, h_twx, nx * sizeof(zd), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(twz, h_twz, nz * sizeof(zd), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(fdw, h_fdw, 5 * ny * sizeof(double), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(fdl0, h_fdl0, ny * sizeof(int), cudaMemcpyHostToDevice, st));
    k_pair_table<<<ny, 128, 0, st>>>(ny, pair_i);
    TRY(cudaStreamSynchronize(st));
    // the array keeps the previous call's contents: clear the sums
    TRY(cudaMemsetAsync(mean_sum, 0, 4 * ny * sizeof(double), st));
    TRY(cudaMemsetAsync(stats, 0, NSTAT * ny * sizeof(double), st));
    TRY(cudaMemsetAsync(nonfinite, 0, sizeof(int), st));

    // Step 1: ensemble mean of this batch
    const zd* f = (const zd*)fields;
    k_mean_accum<<<(4 * ny + 127) / 128, 128, 0, st>>>(f, ns, ny, (long long)Nk, mean_sum);
    k_div<<<(4 * ny + 127) / 128, 128, 0, st>>>(mean_sum, (double)ns, 4 * ny, mean);
    k_profiles<<<(ny + 127) / 128, 128, 0, st>>>(mean_sum, (double)ns, stats, 1.0, (long long)nx * nz, d.nu, 0, fdw, fdl0,
                                                  ny, prof);
    // Step 2: products, contractions, per-pair term spectra
    ProdArgs a;
    a.fields = f; a.ns = ns; a.ny = ny; a.nz = nz; a.nx = nx; a.nxh = nxh; a.Nk = Nk;
    a.mean = mean; a.Xop = Xop; a.G = G; a.H = H; a.tw_x = twx; a.tw_z = twz;
    a.part = part; a.stats = stats; a.nonfinite = nonfinite;
    a.cw_ci = tl.cw_ci; a.rz_rp = tl.rz_rp; a.cw_cf = tl.cw_cf; a.yb_cf = tl.yb_cf; a.eps_kchunk = EPS_KCHUNK;
    a.Lx = d.Lx; a.Lz = d.Lz; a.fdw = fdw; a.fdl0 = fdl0; a.st = st;
    products_launch<double>(a);
    correlate_launch(false, Xop, ns, ny, Nk, 0, Nk, raw, job_set(tset), st);
    combine_launch(false, true, raw, ny, nz, nx, d.Lx, d.Lz, d.nu, prof, 0, 0, Nk, Nk, comb, tset, 0, st);
    // Step 3: profiles, inverse transforms, stencils
    k_profiles<<<(ny + 127) / 128, 128, 0, st>>>(mean_sum, (double)ns, stats, (double)ns, (long long)nx * nz, d.nu, 0, fdw,
                                                  fdl0, ny, prof);
    TermArgs t;
    t.fp32 = false; t.comb64 = true; t.comb = comb; t.W = W; t.pair_i = pair_i; t.npair = npair; t.pair_chunk = npair;
    t.ny = ny; t.nz = nz; t.nx = nx; t.cw = tl.cw_tc; t.rz = tl.rz_tr; t.inv_count = 1.0 / ns; t.prof = prof;
    t.tw_x = twx; t.tw_z = twz; t.terms = terms; t.spec = nullptr; t.sep = full_sep(nz, nx); t.st = st;
    t.tmask = tset;
    terms_launch(t);
    stencil_launch(false, 0, terms, nullptr, npair, pair_i, ny, full_sep(nz, nx), d.nu, fdw, fdl0, prof, tset, st);
    if (profiles) TRY(cudaMemcpyAsync(profiles, prof, GKE_NPROF * ny * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int bad = 0;
    TRY(cudaMemcpyAsync(&bad, nonfinite, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    TRY(cudaGetLastError());
#undef TRY
    if (bad) return fail(GKE_ERR_NONFINITE, "non-finite value in the input");
    return GKE_OK;
}
