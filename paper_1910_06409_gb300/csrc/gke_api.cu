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
#include <unistd.h>
#include <type_traits>
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
    // npair: output pairs (the triangle, or the wedge with mirror sampling);
    // npair_tri: pairs of the triangle, over which the spectra are summed
    long long npair = 0, npair_tri = 0;
    bool wedge = false;
    unsigned tset = 0;                        // terms computed (term_set of the mask)
    int comb_kc = 0;                          // wavenumbers per combine CTA (0 = default; tuner)
    int w_mib = 0;                            // inverse-transform scratch per pair chunk, MiB (tuner)
    int knob_source = 0;                      // 0 built-in, 1 tuning file, 2 measured
    void* fold = nullptr;                     // wedge: folded spectra (aliases raw when it fits)
    bool fold_owned = false;
    // kept separations (undersampling): host lists and the device map
    std::vector<int> keep_z, keep_x;
    SepMap sep;
    int* sep_tab = nullptr;
    // uniform undersampling by (sz, sx) done by spectral aliasing: the
    // contractions run in chunks of whole conjugate classes of kz rows (at
    // most R rows, Kc wavenumbers), each chunk's operands gathered into Xc and
    // its contractions folded into the FP64 coarse spectra of every triangle
    // pair, comb[npair_tri][NTERM][nzd][nxd/2+1] (the wedge's mirror average
    // is formed from them at finalize)
    bool dec = false;
    int nzt = 0, nxt = 0;                     // transform sizes of the terms stage (nzd, nxd when dec)
    int R = 0, Kc = 0;                        // chunk rows and wavenumbers (the largest chunk)
    void* Xc = nullptr;                       // one chunk's gathered operands
    // split path with at most 4 row tiles: the chunk's correlator writes the
    // six plane spectra [NPLANE][Kc][npp] (in raw) and k_planes_fold aliases
    // them; pair_tri lists the triangle's pairs for it
    bool dec_planes = false;
    int* pair_tri = nullptr;
    int* dec_tab = nullptr;                   // per chunk: its kz rows, then its coarse rows
    // Step 1 for velocity-vorticity databases (allocated on first use):
    // transform buffers of six fields, d2/dy2 weights, the factored Poisson
    // operators, staging of host inputs and outputs
    zd *s1_A = nullptr, *s1_B = nullptr, *s1_in = nullptr, *s1_out = nullptr;
    double *s1_w2 = nullptr, *s1_ab = nullptr, *s1_mean = nullptr;
    unsigned char* s1_piv = nullptr;
    bool s1_ready = false;
    // streamed input of gke_compute from pinned host memory: the k = 0
    // coefficients for the Step-1 mean, then whole snapshots on up_st, each
    // announced by up_ev[s] (products_stage passes up_active to the kernels)
    zd* k0buf = nullptr;
    cudaStream_t up_st = nullptr;
    std::vector<cudaEvent_t> up_ev;
    const cudaEvent_t* up_active = nullptr;
    std::vector<int> ch_rows, ch_nrows, ch_crs, ch_ncr;   // offsets into dec_tab and counts
    size_t n_acc = 0;                         // elements of the FP64 accumulator comb
    zd *ttw_xd = nullptr, *ttw_zd = nullptr;  // twiddles of the transform sizes
    zf *ttw_xf = nullptr, *ttw_zf = nullptr;
    // device workspaces; Xop, G, H, raw and W hold complex<TF>, TF = double on
    // the plain path and float on the split path
    void *Xop = nullptr, *G = nullptr, *H = nullptr, *raw = nullptr, *W = nullptr;
    void *G2 = nullptr, *H2 = nullptr;        // second products buffers (odd snapshots)
    double* part2 = nullptr;
    // per-pair term spectra summed over batches: FP64 (comb) on the plain path;
    // on the split path the first batch goes to comb32 and a second batch
    // promotes the sum to FP64 (comb, allocated then)
    zd* comb = nullptr;
    zf* comb32 = nullptr;
    bool comb_is64 = false;
    // split plane mode (BF16 x3, triangle, one 128-row tile): the correlator
    // writes the plane spectra of each batch (pl32, FP32), summed in FP64
    // (pl64) from the second batch on; no raw contractions, no combine
    bool planes = false;
    unsigned pset = 0;                        // planes the term set needs (plane_set)
    long long npp = 0;                        // pairs per plane row: npair rounded up to a multiple of 4
    zf* pl32 = nullptr;
    zd* pl64 = nullptr;
    bool pl_is64 = false;
    float* spec = nullptr;                    // split path: spectral parts of A, Phi_y, phi
    size_t tsz = 8;                           // bytes of one output term value
    zd *tw_xd = nullptr, *tw_zd = nullptr, *stage_in = nullptr;
    zf *tw_xf = nullptr, *tw_zf = nullptr;
    size_t csz = 16;                          // bytes of one complex<TF>
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
    std::vector<double> mean_sum_host;       // staging of the symmetrised mean sums
    // host-output finalize: copies of finished term rows overlap the rest
    cudaStream_t copy_st = nullptr;
    cudaStream_t aux_st = nullptr;            // row passes of the inverse transforms
    cudaEvent_t aux_ev[10] = {};              // events of the two-stream stages (products 6, transforms 4)
    // graph replay (gke_compute_graph): the captured pass and what it was captured for
    cudaGraphExec_t graph = nullptr;
    const void* g_fields = nullptr; void* g_terms = nullptr; double* g_prof = nullptr;
    int g_nsnap = 0;
    long long g_launches = 0;
    void* W2 = nullptr;                       // second transform scratch buffer
    std::vector<cudaEvent_t> chunk_ev;
    void* host_terms = nullptr;
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
// Weights of the derivatives of orders 0..M at z0 on the nodes x[0..n), by
// Fornberg's recursion (B. Fornberg, Math. Comp. 51 (1988) 699-706): c[m*n+i]
// is the weight of node i in the m-th derivative.
static void fornberg(const double* x, int n, double z0, int M, double* c)
{
    for (int i = 0; i < (M + 1) * n; ++i) c[i] = 0.0;
    c[0] = 1.0;
    double c1 = 1.0, c4 = x[0] - z0;
    for (int i = 1; i < n; ++i) {
        const int mn = std::min(i, M);
        double c2 = 1.0;
        const double c5 = c4;
        c4 = x[i] - z0;
        for (int j = 0; j < i; ++j) {
            const double c3 = x[i] - x[j];
            c2 *= c3;
            if (j == i - 1) {
                for (int m = mn; m >= 1; --m) c[m * n + i] = c1 * (m * c[(m - 1) * n + i - 1] - c5 * c[m * n + i - 1]) / c2;
                c[i] = -c1 * c5 * c[i - 1] / c2;
            }
            for (int m = mn; m >= 1; --m) c[m * n + j] = (c4 * c[m * n + j] - m * c[(m - 1) * n + j]) / c3;
            c[j] = c4 * c[j] / c3;
        }
        c1 = c2;
    }
}

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

// bytes of inverse-transform scratch per pair chunk (each of two buffers)
static const long long W_CHUNK_BYTES = 192LL << 20;
// bytes of contractions + per-pair spectra of one wavenumber chunk (chunked mode)
static const size_t DEC_CHUNK_BYTES = (size_t)32 << 30;
// above this size of one batch's contractions the plan runs in the chunked mode
static const size_t CHUNKED_RAW_BYTES = (size_t)96 << 30;


// separation indices kept along one direction (a-posteriori undersampling,
// Sec. 3.4): with d = min(m, n - m), keep d < t1, multiples of s1 for
// t1 <= d < t2 and multiples of s2 from t2 on; {0, 0, 0, 0} keeps all
// stride s when the option keeps exactly the multiples of s (t2 = 0: every d
// multiple of s2), else 0; all zero is stride 1
static int uniform_stride(int n, const int u[4])
{
    if (!u[0] && !u[1] && !u[2] && !u[3]) return 1;
    if (u[0] == 0 && u[1] == 0 && u[3] >= 1 && n % u[3] == 0) return u[3];
    return 0;
}

static bool under_valid(const int u[4])
{
    if (!u[0] && !u[1] && !u[2] && !u[3]) return true;
    return u[0] >= 0 && u[1] >= u[0] && (u[1] == u[0] || u[2] >= 1) && u[3] >= 1;
}
static std::vector<int> kept_indices(int n, const int u[4])
{
    std::vector<int> k;
    const bool all = !u[0] && !u[1] && !u[2] && !u[3];
    for (int m = 0; m < n; ++m) {
        const int d = std::min(m, n - m);
        if (all || d < u[0] || (d < u[1] ? d % u[2] == 0 : d % u[3] == 0)) k.push_back(m);
    }
    return k;
}

static bool is_pinned_host_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeHost;
}

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

static cudaError_t set_smem_attrs()
{
    int lim = smem_limit();
    cudaError_t e = products_set_attrs(lim);
    if (e == cudaSuccess) e = terms_set_attrs(lim);
    if (e == cudaSuccess) e = combine_set_attrs();
    return e;
}

template <typename T> static cudaError_t dalloc(T** p, size_t count)
{
    return cudaMalloc((void**)p, count * sizeof(T));
}

// ------------------------------------------------------------------- plan
// ------------------------------------------------------------- autotuner
// Knobs of the schedule that do not change any result: the pair-chunk size
// of the inverse transforms (scratch W per chunk) and the wavenumbers per
// CTA of the combine kernel.  Tuned per device and problem shape, by timing
// each candidate on the plan's own workspaces, and kept in a text file.
static const int W_MIB_CAND[3] = {48, 96, 192};

static long long pairs_for(const gke_plan_t p, int mib)
{
    const long long per = (long long)NTERM * p->sep.nrz * (p->nxt / 2 + 1) * (long long)p->csz;
    const long long n = std::max<long long>(1, std::min<long long>(p->npair, ((long long)mib << 20) / per));
    return p->planes ? std::max<long long>(4, n & ~3LL) : n;       // plane mode: whole pair groups
}

static std::string tune_key(const gke_plan_t p)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown";
    for (char& c : name)
        if (c == ' ' || c == ':') c = '_';
    const gke_desc& d = p->d;
    char buf[512];
    snprintf(buf, sizeof buf, "gke-tune-1 %s sm%d nx%d nz%d ny%d prec%d dom%d dec%d nzt%d nxt%d nrz%d nrx%d terms%u",
             name.c_str(), nsm, d.nx, d.nz, d.ny, d.precision, d.pair_domain, p->dec ? 1 : 0, p->nzt, p->nxt,
             p->sep.nrz, p->sep.nrx, p->tset);
    return buf;
}

static bool tune_lookup(const char* path, const std::string& key, int& w_mib, int& kc)
{
    FILE* fp = fopen(path, "r");
    if (!fp) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof line, fp)) {
        const std::string l(line);
        const size_t c = l.find(" : ");
        if (c == std::string::npos || l.compare(0, c, key) != 0 || c != key.size()) continue;
        int a = 0, b = 0;
        if (sscanf(l.c_str() + c + 3, "w_mib=%d comb_kc=%d", &a, &b) == 2) { w_mib = a; kc = b; found = true; }
    }
    fclose(fp);
    return found;
}

// The file's lines plus this one go to a private temporary file that is then
// renamed over the tuning file, so processes storing at the same time (replica
// ranks tuning one shape) never interleave partial lines; one of two racing
// stores may be lost, which only means timing that shape again.  Lookups take
// the last valid line of a key.
static void tune_store(const char* path, const std::string& key, int w_mib, int kc)
{
    std::string text;
    if (FILE* in = fopen(path, "r")) {
        char buf[4096];
        size_t n;
        while ((n = fread(buf, 1, sizeof buf, in)) > 0) text.append(buf, n);
        fclose(in);
        if (!text.empty() && text.back() != '\n') text += '\n';
    }
    char line[1024];
    snprintf(line, sizeof line, "%s : w_mib=%d comb_kc=%d\n", key.c_str(), w_mib, kc);
    text += line;
    const std::string tmp = std::string(path) + ".tmp." + std::to_string((long long)getpid());
    FILE* out = fopen(tmp.c_str(), "w");
    if (!out) return;
    const bool ok = fwrite(text.data(), 1, text.size(), out) == text.size();
    if (fclose(out) != 0 || !ok || rename(tmp.c_str(), path) != 0) remove(tmp.c_str());
}

// device time of f() on the plan's stream, the second of two runs
template <typename F>
static float time_twice(gke_plan_t p, F f)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    f();
    cudaEventRecord(a, p->st);
    f();
    cudaEventRecord(b, p->st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

static void terms_stage(gke_plan_t p, void* terms_dev);

// times the candidates on the plan's workspaces (their contents are not yet
// data); each knob is set to its fastest candidate
static gke_status tune_knobs(gke_plan_t p)
{
    const gke_desc& d = p->d;
    const bool f32 = d.precision != GKE_PREC_F64;
    const bool timing0 = p->timing;
    p->timing = false;
    const long long launches = p->launches;
    // combine: one batch's spectra into the first-batch accumulator (plans
    // that combine raw contractions per pair; plane mode and the chunked
    // mode's fused fold keep the default)
    if (p->planes || p->dec) p->comb_kc = combine_kc(f32);
    else {
        const int cand[3] = {f32 ? 2 : 1, f32 ? 4 : 2, f32 ? 8 : 4};
        float best = 0.f;
        for (int kc : cand) {
            const float ms = time_twice(p, [&] {
                combine_launch(f32, p->comb_is64, p->raw, d.ny, d.nz, d.nx, d.Lx, d.Lz, d.nu, p->prof, 0, 0,
                               p->Nk, p->Nk, p->comb_is64 ? (void*)p->comb : (void*)p->comb32, p->tset, kc,
                               p->st);
            });
            if (p->comb_kc == 0 || ms < best) { best = ms; p->comb_kc = kc; }
        }
    }
    // inverse transforms of the first pairs (two chunks of the largest
    // candidate) into a scratch output
    const long long P = std::min<long long>(p->npair, 2 * pairs_for(p, W_MIB_CAND[2]));
    if (P > pairs_for(p, W_MIB_CAND[0])) {
        const long long N = (long long)p->sep.nrz * p->sep.nrx;
        void* out = nullptr;
        float* spec = nullptr;
        if (cudaMalloc(&out, (size_t)NTERM * P * N * p->tsz) != cudaSuccess ||
            (f32 && cudaMalloc((void**)&spec, (size_t)3 * P * N * sizeof(float)) != cudaSuccess)) {
            if (out) cudaFree(out);
            cudaGetLastError();
            p->w_mib = W_MIB_CAND[2];           // no room to time it: the built-in chunk
            p->pair_chunk = pairs_for(p, p->w_mib);
            p->launches = launches;
            p->timing = timing0;
            return GKE_OK;
        }
        const long long npair = p->npair;
        float* spec0 = p->spec;
        const double cnt = p->snap_count;
        p->npair = P;                            // terms_stage indexes outputs by npair
        p->spec = spec;
        p->snap_count = 1.0;
        float best = 0.f;
        for (int mib : W_MIB_CAND) {
            p->pair_chunk = pairs_for(p, mib);
            const float ms = time_twice(p, [&] { terms_stage(p, out); });
            if (p->w_mib == 0 || ms < best) { best = ms; p->w_mib = mib; }
        }
        p->npair = npair;
        p->spec = spec0;
        p->snap_count = cnt;
        cudaStreamSynchronize(p->st);
        cudaFree(out);
        if (spec) cudaFree(spec);
    } else {
        p->w_mib = W_MIB_CAND[2];
    }
    p->pair_chunk = pairs_for(p, p->w_mib);
    p->launches = launches;
    p->timing = timing0;
    CUDA_TRY(p, cudaGetLastError());
    return GKE_OK;
}

extern "C" gke_status gke_plan_knobs(gke_plan_t p, int* w_chunk_mib, int* comb_kc, int* source)
{
    if (!p) return GKE_ERR_ARG;
    if (w_chunk_mib) *w_chunk_mib = p->w_mib ? p->w_mib : (int)(W_CHUNK_BYTES >> 20);
    if (comb_kc) *comb_kc = p->comb_kc ? p->comb_kc : combine_kc(p->d.precision != GKE_PREC_F64);
    if (source) *source = p->knob_source;
    return GKE_OK;
}

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
    if (!fft_len_ok(d.nx) || !fft_len_ok(d.nz)) {
        g_plan_err = "nx and nz must be 2^a or 3 * 2^a (transform lengths of the library)";
        return GKE_ERR_UNSUPPORTED;
    }
    if (d.precision != GKE_PREC_F64 && d.precision != GKE_PREC_BF16X3 && d.precision != GKE_PREC_F32) {
        g_plan_err = "unknown precision";
        return GKE_ERR_ARG;
    }
    if (d.pair_domain != GKE_DOMAIN_TRIANGLE && d.pair_domain != GKE_DOMAIN_WEDGE) {
        g_plan_err = "unknown pair_domain";
        return GKE_ERR_ARG;
    }
    if (!under_valid(d.under_x) || !under_valid(d.under_z)) {
        g_plan_err = "undersampling {t1, t2, s1, s2} needs 0 <= t1 <= t2, s2 >= 1, s1 >= 1 if t1 < t2 (or all zero)";
        return GKE_ERR_ARG;
    }
    if (d.term_mask & ~GKE_ALL_TERMS) { g_plan_err = "term_mask has bits above GKE_NTERM"; return GKE_ERR_ARG; }
    for (int j = 1; j < d.ny; ++j)
        if (!(d.y[j] > d.y[j - 1])) { g_plan_err = "y must be strictly increasing"; return GKE_ERR_ARG; }
    if (d.pair_domain == GKE_DOMAIN_WEDGE) {
        // mirror sampling needs a grid symmetric about the centreline
        const double c = d.y[0] + d.y[d.ny - 1], tol = 1e-12 * (d.y[d.ny - 1] - d.y[0]);
        for (int j = 0; j < d.ny; ++j)
            if (std::fabs(d.y[j] + d.y[d.ny - 1 - j] - c) > tol) {
                g_plan_err = "pair_domain GKE_DOMAIN_WEDGE needs a y grid symmetric about its centre";
                return GKE_ERR_ARG;
            }
    }

    gke_plan_t p = new (std::nothrow) gke_plan_s;
    if (!p) { g_plan_err = "host allocation failed"; return GKE_ERR_OOM; }
    p->d = d;
    p->tset = term_set(d.term_mask);
    p->y.assign(d.y, d.y + d.ny);
    p->d.y = p->y.data();
    p->st = (cudaStream_t)stream;
    p->nxh = d.nx / 2 + 1;
    p->Nk = d.nz * p->nxh;
    p->npair_tri = (long long)d.ny * (d.ny + 1) / 2;
    p->wedge = (d.pair_domain == GKE_DOMAIN_WEDGE);
    p->npair = p->npair_tri;
    if (p->wedge) {
        p->npair = 0;
        for (int i1 = 0; 2 * i1 <= d.ny - 1; ++i1) p->npair += d.ny - 2 * i1;
    }
    const int ny = d.ny, ns = d.max_snap, Nk = p->Nk;
    const size_t plane = (size_t)d.nz * p->nxh;
    p->keep_z = kept_indices(d.nz, d.under_z);
    p->keep_x = kept_indices(d.nx, d.under_x);
    const int nrz = (int)p->keep_z.size(), nrx = (int)p->keep_x.size();
    bool under = nrz < d.nz || nrx < d.nx;
    p->sep = full_sep(d.nz, d.nx);
    p->sep.nrz = nrz;
    p->sep.nrx = nrx;
    p->nzt = d.nz;
    p->nxt = d.nx;
    {
        // the chunked mode: under a uniform stride, or when one batch's
        // contractions for all wavenumbers would exceed CHUNKED_RAW_BYTES
        const int sz = uniform_stride(d.nz, d.under_z), sx = uniform_stride(d.nx, d.under_x);
        const size_t raw_all = (size_t)NJOB * ((ny + 7) / 8) * ((ny + 7) / 8) * 64 * (size_t)Nk *
                               (d.precision == GKE_PREC_F64 ? sizeof(zd) : sizeof(zf));
        if (sz && sx && (sz > 1 || sx > 1 || raw_all > CHUNKED_RAW_BYTES) && d.nz / sz >= 4 && d.nx / sx >= 4) {
            p->dec = true;
            p->nzt = d.nz / sz;
            p->nxt = d.nx / sx;
            p->sep = full_sep(p->nzt, p->nxt);     // the coarse grid is stored whole
            under = false;
        }
    }

    // the split correlator writes the term planes directly when the wall-normal
    // rows fit one 128-row tile (the full triangle; the wedge and the chunked
    // mode combine raw contractions)
    p->planes = d.precision == GKE_PREC_BF16X3 && !p->dec && !p->wedge && split_planes_ok(ny);
    p->pset = plane_set(p->tset);
    auto bail = [&](gke_status s, const std::string& m) { g_plan_err = m; gke_destroy(p); return s; };
    cudaError_t e;
#define ALLOC(ptr, n)                                                                          \
    do {                                                                                       \
        e = dalloc(&(ptr), (size_t)(n));                                                       \
        if (e != cudaSuccess) return bail(GKE_ERR_OOM, std::string("cudaMalloc " #ptr ": ") +  \
                                                           cudaGetErrorString(e));             \
    } while (0)
    const bool f32 = (d.precision != GKE_PREC_F64);
    p->csz = f32 ? sizeof(zf) : sizeof(zd);
#define ALLOCB(ptr, bytes)                                                                          \
    do {                                                                                            \
        e = cudaMalloc((void**)&(ptr), (size_t)(bytes));                                            \
        if (e != cudaSuccess) return bail(GKE_ERR_OOM, std::string("cudaMalloc " #ptr ": ") +       \
                                                           cudaGetErrorString(e));                  \
    } while (0)
    ALLOCB(p->Xop, (size_t)NFIELD * Nk * ns * ny * p->csz);
    ALLOCB(p->G, (size_t)4 * ny * plane * p->csz);
    ALLOCB(p->H, (size_t)7 * ny * plane * p->csz);
    ALLOCB(p->G2, (size_t)4 * ny * plane * p->csz);
    ALLOCB(p->H2, (size_t)7 * ny * plane * p->csz);
    const size_t raw_per_k = (size_t)NJOB * ((ny + 7) / 8) * ((ny + 7) / 8) * 64 * p->csz;
    if (p->dec) {
        // conjugate classes of kz rows, {kz : kz mod nzd in {c, nzd - c}},
        // c = 0 .. nzd/2, packed in order into chunks of at most R rows; R
        // keeps a chunk's contractions and gathered operands within
        // DEC_CHUNK_BYTES, but a chunk holds at least one class
        const int nzd = p->nzt;
        p->dec_planes = d.precision == GKE_PREC_BF16X3 && split_planes_ok(ny);
        p->npp = 4 * ((p->npair_tri + 3) / 4);
        const size_t chunk_per_k = p->dec_planes ? (size_t)NPLANE * p->npp * sizeof(zf) : raw_per_k;
        const size_t per_row = (size_t)p->nxh * (chunk_per_k + (size_t)NFIELD * ns * ny * p->csz);
        p->R = (int)std::max<size_t>((size_t)2 * (d.nz / nzd), DEC_CHUNK_BYTES / per_row);
        std::vector<int> tab;
        std::vector<int> rows, crs;
        auto close_chunk = [&]() {
            if (rows.empty()) return;
            p->ch_rows.push_back((int)tab.size());
            p->ch_nrows.push_back((int)rows.size());
            tab.insert(tab.end(), rows.begin(), rows.end());
            p->ch_crs.push_back((int)tab.size());
            p->ch_ncr.push_back((int)crs.size());
            tab.insert(tab.end(), crs.begin(), crs.end());
            rows.clear();
            crs.clear();
        };
        int rmax = 0;
        for (int c = 0; c <= nzd / 2; ++c) {
            const int c2 = (nzd - c) % nzd;
            std::vector<int> cls;
            for (int kz = 0; kz < d.nz; ++kz)
                if (kz % nzd == c || kz % nzd == c2) cls.push_back(kz);
            if (!rows.empty() && rows.size() + cls.size() > (size_t)p->R) close_chunk();
            rows.insert(rows.end(), cls.begin(), cls.end());
            crs.push_back(c);
            if (c2 != c) crs.push_back(c2);
            rmax = std::max(rmax, (int)rows.size());
        }
        close_chunk();
        p->R = rmax;
        p->Kc = p->R * p->nxh;
        ALLOCB(p->raw, chunk_per_k * p->Kc);
        if (p->dec_planes && p->wedge) ALLOCB(p->pair_tri, (size_t)2 * p->npair_tri * sizeof(int));
        ALLOCB(p->Xc, (size_t)NFIELD * p->Kc * ns * ny * p->csz);
        ALLOCB(p->dec_tab, tab.size() * sizeof(int));
        if ((e = cudaMemcpy(p->dec_tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(GKE_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
        const size_t ncoarse = (size_t)p->nzt * (p->nxt / 2 + 1);
        p->n_acc = (size_t)p->npair_tri * NTERM * ncoarse;
        ALLOC(p->comb, p->n_acc);
        if (p->wedge) {
            ALLOCB(p->fold, (size_t)p->npair * NTERM * ncoarse * sizeof(zd));
            p->fold_owned = true;
        }
        p->tsz = f32 ? sizeof(float) : sizeof(double);
        if (f32) ALLOC(p->spec, (size_t)3 * p->npair * p->nxt * p->nzt + 15 * (size_t)p->npair);
    } else if (p->planes) {
        // the six plane spectra of one batch, [NPLANE][Nk][npp]
        p->Kc = Nk;
        p->npp = 4 * ((p->npair_tri + 3) / 4);
        p->n_acc = (size_t)NPLANE * Nk * p->npp;
        ALLOC(p->pl32, p->n_acc);
        ALLOC(p->spec, (size_t)3 * p->npair * nrx * nrz + 15 * (size_t)p->npair);
        p->tsz = sizeof(float);
    } else {
    p->Kc = Nk;
    p->n_acc = (size_t)p->npair_tri * NTERM * Nk;
    const size_t raw_bytes = raw_per_k * Nk;
    ALLOCB(p->raw, raw_bytes);
    if (p->wedge) {
        // the folded spectra of the output pairs (at most complex128) are
        // formed at finalize, when raw is free
        const size_t fold_bytes = (size_t)p->npair * NTERM * Nk * sizeof(zd);
        if (fold_bytes <= raw_bytes) p->fold = p->raw;
        else { ALLOCB(p->fold, fold_bytes); p->fold_owned = true; }
    }
    if (f32) {
        ALLOC(p->comb32, (size_t)p->npair_tri * NTERM * Nk);
        // spectral parts of A, Phi_y, phi, then 15 per-pair stencil scalars
        ALLOC(p->spec, (size_t)3 * p->npair * nrx * nrz + 15 * (size_t)p->npair);
        p->tsz = sizeof(float);
    } else {
        ALLOC(p->comb, (size_t)p->npair_tri * NTERM * Nk);
        p->comb_is64 = true;
        p->tsz = sizeof(double);
    }
    }
    // pairs per inverse-transform chunk (W_CHUNK_BYTES of scratch W, two
    // buffers): the column pass of one chunk overlaps the row pass of the
    // previous one on the auxiliary stream
    const int nxth = p->nxt / 2 + 1, nrzt = p->sep.nrz;
    p->pair_chunk = pairs_for(p, (int)(W_CHUNK_BYTES >> 20));
    (void)nxth; (void)nrzt;
    ALLOCB(p->W, (size_t)p->pair_chunk * NTERM * nrzt * nxth * p->csz);
    ALLOCB(p->W2, (size_t)p->pair_chunk * NTERM * nrzt * nxth * p->csz);
    if ((e = cudaStreamCreateWithFlags(&p->aux_st, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(GKE_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    for (cudaEvent_t& ev : p->aux_ev)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return bail(GKE_ERR_CUDA, std::string("event: ") + cudaGetErrorString(e));
    ALLOC(p->tw_xd, d.nx);
    ALLOC(p->tw_zd, d.nz);
    ALLOC(p->tw_xf, d.nx);
    ALLOC(p->tw_zf, d.nz);
    if (p->dec) {
        ALLOC(p->ttw_xd, p->nxt);
        ALLOC(p->ttw_zd, p->nzt);
        ALLOC(p->ttw_xf, p->nxt);
        ALLOC(p->ttw_zf, p->nzt);
    } else {
        p->ttw_xd = p->tw_xd; p->ttw_zd = p->tw_zd; p->ttw_xf = p->tw_xf; p->ttw_zf = p->tw_zf;
    }
#undef ALLOCB
    ALLOC(p->mean_sum, 4 * ny);
    ALLOC(p->mean, 4 * ny);
    ALLOC(p->stats, NSTAT * ny);
    ALLOC(p->prof, NPR * ny);
    ALLOC(p->fdw, 5 * ny);
    ALLOC(p->fdl0, ny);
    ALLOC(p->pair_i, 2 * p->npair);
    ALLOC(p->nonfinite, 1);
    if (under) ALLOC(p->sep_tab, (size_t)d.nz + d.nx + nrz + nrx);
    {
        p->part_count = part_count(d.nz, ny, Nk, pick_tiles(d.nx, d.nz, p->csz));
        ALLOC(p->part, p->part_count);
        ALLOC(p->part2, p->part_count);
    }
    if (d.precision == GKE_PREC_BF16X3) {
        gke_status s = split_alloc(p->split, ny, ns, p->Kc);
        if (s != GKE_OK) return bail(s, "split workspace allocation failed");
    }
#undef ALLOC
    // host tables
    // twiddles e^{-2 pi i m / n}, m < n, from the host's libm in FP64
    std::vector<zd> twx(d.nx), twz(d.nz);
    std::vector<zf> twxf(d.nx), twzf(d.nz);
    for (int m = 0; m < d.nx; ++m) { twx[m].x = std::cos(2.0 * M_PI * m / d.nx); twx[m].y = -std::sin(2.0 * M_PI * m / d.nx); }
    for (int m = 0; m < d.nz; ++m) { twz[m].x = std::cos(2.0 * M_PI * m / d.nz); twz[m].y = -std::sin(2.0 * M_PI * m / d.nz); }
    for (int m = 0; m < d.nx; ++m) { twxf[m].x = (float)twx[m].x; twxf[m].y = (float)twx[m].y; }
    for (int m = 0; m < d.nz; ++m) { twzf[m].x = (float)twz[m].x; twzf[m].y = (float)twz[m].y; }
    std::vector<double> w(5 * ny);
    std::vector<int> l0(ny);
    for (int j = 0; j < ny; ++j) {
        int a = std::min(std::max(j - 2, 0), ny - 5);
        l0[j] = a;
        fornberg_d1(p->y.data() + a, 5, p->y[j], w.data() + 5 * j);
    }
    // output pair table, row-major: the triangle, or the wedge i1 + i2 <= ny - 1
    std::vector<int> pi(2 * p->npair);
    long long q = 0;
    for (int i1 = 0; i1 < ny; ++i1)
        for (int i2 = i1; i2 < (p->wedge ? ny - i1 : ny); ++i2) { pi[2 * q] = i1; pi[2 * q + 1] = i2; ++q; }
    cudaStream_t st = p->st;
    if (p->pair_tri) {
        // the triangle's pairs (the plane fold of the chunked wedge runs over all of them)
        std::vector<int> pt(2 * p->npair_tri);
        long long r = 0;
        for (int i1 = 0; i1 < ny; ++i1)
            for (int i2 = i1; i2 < ny; ++i2) { pt[2 * r] = i1; pt[2 * r + 1] = i2; ++r; }
        if ((e = cudaMemcpy(p->pair_tri, pt.data(), pt.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(GKE_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    std::vector<int> stab;
    if (under) {
        // [zpos (nz) | xpos (nx) | negz (nrz) | negx (nrx)]
        std::vector<int> zpos(d.nz, -1), xpos(d.nx, -1);
        for (int i = 0; i < nrz; ++i) zpos[p->keep_z[i]] = i;
        for (int i = 0; i < nrx; ++i) xpos[p->keep_x[i]] = i;
        stab.insert(stab.end(), zpos.begin(), zpos.end());
        stab.insert(stab.end(), xpos.begin(), xpos.end());
        for (int i = 0; i < nrz; ++i) stab.push_back(zpos[(d.nz - p->keep_z[i]) % d.nz]);
        for (int i = 0; i < nrx; ++i) stab.push_back(xpos[(d.nx - p->keep_x[i]) % d.nx]);
        p->sep.zpos = p->sep_tab;
        p->sep.xpos = p->sep_tab + d.nz;
        p->sep.negz = p->sep_tab + d.nz + d.nx;
        p->sep.negx = p->sep_tab + d.nz + d.nx + nrz;
        if ((e = cudaMemcpyAsync(p->sep_tab, stab.data(), stab.size() * sizeof(int), cudaMemcpyHostToDevice, st)))
            return bail(GKE_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    if (p->dec) {
        // twiddles of the coarse transforms: every s-th entry of the fine ones
        const int sx = d.nx / p->nxt, sz = d.nz / p->nzt;
        std::vector<zd> cx(p->nxt), cz(p->nzt);
        std::vector<zf> cxf(p->nxt), czf(p->nzt);
        for (int m = 0; m < p->nxt; ++m) { cx[m] = twx[m * sx]; cxf[m] = twxf[m * sx]; }
        for (int m = 0; m < p->nzt; ++m) { cz[m] = twz[m * sz]; czf[m] = twzf[m * sz]; }
        if ((e = cudaMemcpyAsync(p->ttw_xd, cx.data(), cx.size() * sizeof(zd), cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(p->ttw_zd, cz.data(), cz.size() * sizeof(zd), cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(p->ttw_xf, cxf.data(), cxf.size() * sizeof(zf), cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(p->ttw_zf, czf.data(), czf.size() * sizeof(zf), cudaMemcpyHostToDevice, st)) ||
            (e = cudaStreamSynchronize(st)))
            return bail(GKE_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(p->tw_xd, twx.data(), twx.size() * sizeof(zd), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(p->tw_zd, twz.data(), twz.size() * sizeof(zd), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(p->tw_xf, twxf.data(), twxf.size() * sizeof(zf), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(p->tw_zf, twzf.data(), twzf.size() * sizeof(zf), cudaMemcpyHostToDevice, st)) ||
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
    if (d.tune_cache) {
        // the schedule: from the tuning file, else measured now and stored
        const std::string key = tune_key(p);
        int w = 0, kc = 0;
        const bool hit = tune_lookup(d.tune_cache, key, w, kc) &&
                         (w == W_MIB_CAND[0] || w == W_MIB_CAND[1] || w == W_MIB_CAND[2]) &&
                         combine_kc_ok(d.precision != GKE_PREC_F64, kc);
        if (hit) {
            p->w_mib = w;
            p->comb_kc = kc;
            p->pair_chunk = pairs_for(p, w);
            p->knob_source = 1;
        } else {
            gke_status ts = tune_knobs(p);
            if (ts != GKE_OK) return bail(ts, p->err);
            tune_store(d.tune_cache, key, p->w_mib, p->comb_kc);
            p->knob_source = 2;
        }
    }
    p->d.tune_cache = nullptr;                  // the caller's string is read during gke_plan only
    gke_status rs = gke_reset(p);
    if (rs != GKE_OK) return bail(rs, p->err);
    *out = p;
    return GKE_OK;
}

extern "C" unsigned gke_term_set(unsigned term_mask) { return term_set(term_mask & GKE_ALL_TERMS); }

extern "C" gke_status gke_reset(gke_plan_t p)
{
    if (!p) return GKE_ERR_ARG;
    CUDA_TRY(p, cudaMemsetAsync(p->mean_sum, 0, 4 * p->d.ny * sizeof(double), p->st));
    CUDA_TRY(p, cudaMemsetAsync(p->stats, 0, NSTAT * p->d.ny * sizeof(double), p->st));
    CUDA_TRY(p, cudaMemsetAsync(p->nonfinite, 0, sizeof(int), p->st));
    p->mean_count = 0.0;
    p->snap_count = 0.0;
    p->mean_frozen = p->have_acc = p->finalized = false;
    p->comb_is64 = (p->d.precision == GKE_PREC_F64) || p->dec;
    p->pl_is64 = false;
    if (p->dec) CUDA_TRY(p, cudaMemsetAsync(p->comb, 0, p->n_acc * sizeof(zd), p->st));
    return GKE_OK;
}

extern "C" void gke_destroy(gke_plan_t p)
{
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st); else cudaDeviceSynchronize();
    if (p->fold_owned) cudaFree(p->fold);
    if (p->W2) cudaFree(p->W2);
    {
        void* more[] = {p->G2, p->H2, p->part2};
        for (void* q : more) if (q) cudaFree(q);
    }
    if (p->aux_st) cudaStreamDestroy(p->aux_st);
    for (cudaEvent_t ev : p->aux_ev) if (ev) cudaEventDestroy(ev);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->dec) {
        void* extra[] = {p->Xc, p->dec_tab, p->pair_tri, p->ttw_xd, p->ttw_zd, p->ttw_xf, p->ttw_zf};
        for (void* q : extra) if (q) cudaFree(q);
    }
    void* s1[] = {p->s1_A, p->s1_B, p->s1_in, p->s1_out, p->s1_w2, p->s1_ab, p->s1_mean, p->s1_piv, p->k0buf};
    for (void* q : s1) if (q) cudaFree(q);
    for (cudaEvent_t e : p->up_ev) cudaEventDestroy(e);
    if (p->up_st) cudaStreamDestroy(p->up_st);
    void* ptrs[] = {p->pl32, p->pl64, p->Xop, p->G, p->H, p->raw, p->comb, p->comb32, p->spec, p->W, p->tw_xd, p->tw_zd, p->tw_xf, p->tw_zf, p->stage_in,
                    p->mean_sum, p->mean, p->stats, p->prof, p->fdw, p->stage_terms, p->stage_prof,
                    p->fdl0, p->pair_i, p->nonfinite, p->part, p->sep_tab};
    for (void* q : ptrs) if (q) cudaFree(q);
    split_free(p->split);
    for (auto& m : p->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
    for (auto e : p->chunk_ev) cudaEventDestroy(e);
    if (p->copy_st) cudaStreamDestroy(p->copy_st);
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
    return p ? (long long)NTERM * p->npair * p->sep.nrx * p->sep.nrz * (long long)p->tsz : -1;
}

extern "C" gke_status gke_separation_labels(gke_plan_t p, int* nrz, int* nrx, int* mz, int* mx)
{
    if (!p) return GKE_ERR_ARG;
    if (nrz) *nrz = p->sep.nrz;
    if (nrx) *nrx = p->sep.nrx;
    if (mz) std::copy(p->keep_z.begin(), p->keep_z.end(), mz);
    if (mx) std::copy(p->keep_x.begin(), p->keep_x.end(), mx);
    return GKE_OK;
}

extern "C" gke_status gke_pair_labels(gke_plan_t p, double* Y, double* ry, int* i1, int* i2)
{
    if (!p) return GKE_ERR_ARG;
    long long q = 0;
    for (int a = 0; a < p->d.ny; ++a)
        for (int b = a; b < (p->wedge ? p->d.ny - a : p->d.ny); ++b, ++q) {
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

// plane: elements between consecutive (snapshot, field, y) rows of f (Nk for
// whole snapshots, 1 for a compact copy of the k = 0 coefficients)
static gke_status mean_impl(gke_plan_t p, const zd* f, int nsnap, long long plane = -1)
{
    const int ny = p->d.ny;
    {
        StageScope sc(p, GKE_STAGE_MEAN);
        k_mean_accum<<<(4 * ny + 127) / 128, 128, 0, p->st>>>(f, nsnap, ny, plane < 0 ? (long long)p->Nk : plane,
                                                              p->mean_sum);
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

static void products_stage(gke_plan_t p, const zd* f, int ns)
{
    const gke_desc& d = p->d;
    const bool f32 = (d.precision != GKE_PREC_F64);
    const Tiles t = pick_tiles(d.nx, d.nz, p->csz);
    ProdArgs a;
    a.fields = f; a.ns = ns; a.ny = d.ny; a.nz = d.nz; a.nx = d.nx; a.nxh = p->nxh; a.Nk = p->Nk;
    a.mean = p->mean; a.Xop = p->Xop; a.G = p->G; a.H = p->H;
    a.tw_x = f32 ? (const void*)p->tw_xf : (const void*)p->tw_xd;
    a.tw_z = f32 ? (const void*)p->tw_zf : (const void*)p->tw_zd;
    a.part = p->part; a.stats = p->stats; a.nonfinite = p->nonfinite;
    a.cw_ci = t.cw_ci; a.rz_rp = t.rz_rp; a.cw_cf = t.cw_cf; a.yb_cf = t.yb_cf; a.eps_kchunk = EPS_KCHUNK;
    a.Lx = d.Lx; a.Lz = d.Lz; a.fdw = p->fdw; a.fdl0 = p->fdl0; a.st = p->st;
    a.st2 = p->aux_st; a.G2 = p->G2; a.H2 = p->H2; a.part2 = p->part2; a.ev = p->aux_ev;
    a.up_ev = p->up_active;
    p->launches += f32 ? products_launch<float>(a) : products_launch<double>(a);
}

static gke_status enqueue_snapshot(gke_plan_t p, const zd* f, int ns);

static gke_status snapshot_impl(gke_plan_t p, const zd* f, int ns)
{
    const gke_desc& d = p->d;
    const int ny = d.ny;
    cudaStream_t st = p->st;
    if (!p->mean_frozen) {
        // mean = mean_sum / mean_count, computed once (host round trip of 4 ny doubles)
        std::vector<double> m(4 * ny);
        CUDA_TRY(p, cudaMemcpyAsync(m.data(), p->mean_sum, m.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(p, cudaStreamSynchronize(st));
        for (double& v : m) v /= p->mean_count;
        if (p->wedge) {
            // the ensemble of snapshots and mirror images: U, W, P even about
            // the centreline, V odd
            std::vector<double> ms(m.size());
            for (int f = 0; f < 4; ++f)
                for (int j = 0; j < ny; ++j)
                    ms[f * ny + j] = 0.5 * (m[f * ny + j] + (f == 1 ? -1.0 : 1.0) * m[f * ny + ny - 1 - j]);
            m.swap(ms);
            p->mean_sum_host.assign(m.size(), 0.0);
            for (size_t i = 0; i < m.size(); ++i) p->mean_sum_host[i] = m[i] * p->mean_count;
            CUDA_TRY(p, cudaMemcpyAsync(p->mean_sum, p->mean_sum_host.data(), m.size() * sizeof(double),
                                        cudaMemcpyHostToDevice, st));
        }
        CUDA_TRY(p, cudaMemcpyAsync(p->mean, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        // U and U' rows of the profiles, used by the term combinations
        k_profiles<<<(ny + 127) / 128, 128, 0, st>>>(p->mean_sum, p->mean_count, p->stats, 1.0,
                                                      (long long)d.nx * d.nz, d.nu, p->wedge ? 1 : 0, p->fdw, p->fdl0, ny, p->prof);
        p->launches += 1;
        CUDA_TRY(p, cudaStreamSynchronize(st));
        p->mean_frozen = true;
    }
    return enqueue_snapshot(p, f, ns);
}

// the kernels of one batch after the mean is frozen (no host synchronisation)
static gke_status enqueue_snapshot(gke_plan_t p, const zd* f, int ns)
{
    const gke_desc& d = p->d;
    const int ny = d.ny, Nk = p->Nk;
    cudaStream_t st = p->st;
    const bool f32 = (d.precision != GKE_PREC_F64);
    {
        StageScope sc(p, GKE_STAGE_PRODUCTS);
        products_stage(p, f, ns);
    }
    // contractions of the wavenumbers [k0, k0 + Kc) of the operand set X
    // (NkX wavenumbers) into raw
    auto correlate = [&](const void* X, int NkX, int k0, int Kc) -> gke_status {
        StageScope sc(p, GKE_STAGE_CORRELATE);
        if (d.precision != GKE_PREC_BF16X3) {
            correlate_launch(f32, X, ns, ny, NkX, k0, Kc, p->raw, job_set(p->tset), st);
            p->launches += 1;
            return GKE_OK;
        }
        int nl = 0;
        gke_status s = split_correlate(p->split, (const zf*)X, ns, ny, NkX, k0, Kc, (zf*)p->raw, job_set(p->tset),
                                       st, p->err, &nl);
        p->launches += nl;
        return s;
    };
    if (p->dec) {
        // chunks of conjugate row classes: the chunk's operands gathered, its
        // contractions, and their fused combine + aliasing fold into the FP64
        // coarse spectra of every triangle pair
        for (size_t c = 0; c < p->ch_nrows.size(); ++c) {
            const int nr = p->ch_nrows[c], Kc = nr * p->nxh;
            const int* rows = p->dec_tab + p->ch_rows[c];
            {
                StageScope sc(p, GKE_STAGE_CORRELATE);
                p->launches += gather_rows_launch(!f32, p->Xop, NFIELD, Nk, (long long)ns * ny, rows, nr, p->nxh,
                                                  p->Xc, st);
            }
            if (p->dec_planes) {
                {
                    StageScope sc(p, GKE_STAGE_CORRELATE);
                    int nl = 0;
                    gke_status s = split_correlate_planes(p->split, (const zf*)p->Xc, ns, ny, Kc, 0, Kc, p->pset,
                                                          p->npp, p->prof, (zf*)p->raw, st, p->err, &nl);
                    p->launches += nl;
                    if (s != GKE_OK) return s;
                }
                StageScope sc(p, GKE_STAGE_COMBINE);
                p->launches += planes_fold_launch(p->raw, p->npp, Kc, rows, nr, p->dec_tab + p->ch_crs[c],
                                                  p->ch_ncr[c], p->pair_tri ? p->pair_tri : p->pair_i, p->npair_tri,
                                                  ny, d.nz, d.nx, p->nzt, p->nxt, d.Lx, d.Lz, d.nu, p->prof, p->tset,
                                                  p->comb, st);
                continue;
            }
            gke_status s = correlate(p->Xc, Kc, 0, Kc);
            if (s != GKE_OK) return s;
            StageScope sc(p, GKE_STAGE_COMBINE);
            p->launches += combine_fold_launch(!f32, p->raw, rows, nr, p->dec_tab + p->ch_crs[c], p->ch_ncr[c], ny,
                                               d.nz, d.nx, p->nzt, p->nxt, d.Lx, d.Lz, d.nu, p->prof, p->tset,
                                               p->comb, st);
        }
        CUDA_TRY(p, cudaGetLastError());
        p->snap_count += ns;
        p->have_acc = true;
        return GKE_OK;
    }
    if (p->planes) {
        const long long per_plane = (long long)Nk * p->npp;
        if (p->have_acc && !p->pl_is64) {
            // second batch: the first batch's planes to the FP64 sums first
            StageScope sc(p, GKE_STAGE_COMBINE);
            if (!p->pl64) CUDA_TRY(p, dalloc(&p->pl64, p->n_acc));
            p->launches += planes_accum_launch(p->pl32, per_plane, p->pset, 0, p->pl64, st);
            p->pl_is64 = true;
        }
        {
            StageScope sc(p, GKE_STAGE_CORRELATE);
            int nl = 0;
            gke_status s = split_correlate_planes(p->split, (const zf*)p->Xop, ns, ny, Nk, 0, Nk, p->pset, p->npp,
                                                  p->prof, p->pl32, st, p->err, &nl);
            p->launches += nl;
            if (s != GKE_OK) return s;
        }
        if (p->pl_is64) {
            StageScope sc(p, GKE_STAGE_COMBINE);
            p->launches += planes_accum_launch(p->pl32, per_plane, p->pset, 1, p->pl64, st);
        }
        CUDA_TRY(p, cudaGetLastError());
        p->snap_count += ns;
        p->have_acc = true;
        return GKE_OK;
    }
    {
        gke_status s = correlate(p->Xop, Nk, 0, Nk);
        if (s != GKE_OK) return s;
    }
    {
        StageScope sc(p, GKE_STAGE_COMBINE);
        const long long ncomb = p->npair_tri * NTERM * (long long)Nk;
        if (f32 && p->have_acc && !p->comb_is64) {
            // second batch on the split path: promote the per-pair sums to FP64
            if (!p->comb) CUDA_TRY(p, dalloc(&p->comb, (size_t)ncomb));
            p->launches += promote_launch(p->comb32, ncomb, p->comb, st);
            p->comb_is64 = true;
        }
        void* dst = p->comb_is64 ? (void*)p->comb : (void*)p->comb32;
        p->launches += combine_launch(f32, p->comb_is64, p->raw, d.ny, d.nz, d.nx, d.Lx, d.Lz, d.nu, p->prof,
                                      p->have_acc ? 1 : 0, 0, Nk, Nk, dst, p->tset, p->comb_kc, st);
    }
    CUDA_TRY(p, cudaGetLastError());
    p->snap_count += ns;
    p->have_acc = true;
    return GKE_OK;
}

extern "C" gke_status gke_velocity_vorticity(gke_plan_t p, const void* v_eta, const double* mean_uw, int nsnap,
                                              void* fields)
{
    if (!p || !v_eta || !mean_uw || !fields)
        return p ? fail(p, GKE_ERR_ARG, "v_eta, mean_uw or fields is NULL") : GKE_ERR_ARG;
    if (nsnap < 1) return fail(p, GKE_ERR_ARG, "nsnap < 1");
    const gke_desc& d = p->d;
    const int ny = d.ny;
    const long long fs = (long long)ny * p->Nk;
    cudaStream_t st = p->st;
    if (!p->s1_ready) {
        // workspaces, the d2/dy2 weights and the factored Poisson operators
        if (!p->s1_A) CUDA_TRY(p, cudaMalloc((void**)&p->s1_A, (size_t)6 * fs * sizeof(zd)));
        if (!p->s1_B) CUDA_TRY(p, cudaMalloc((void**)&p->s1_B, (size_t)6 * fs * sizeof(zd)));
        if (!p->s1_w2) CUDA_TRY(p, cudaMalloc((void**)&p->s1_w2, (size_t)5 * ny * sizeof(double)));
        if (!p->s1_mean) CUDA_TRY(p, cudaMalloc((void**)&p->s1_mean, (size_t)2 * ny * sizeof(double)));
        if (!p->s1_piv) CUDA_TRY(p, cudaMalloc((void**)&p->s1_piv, (size_t)fs));
        if (!p->s1_ab) CUDA_TRY(p, cudaMalloc((void**)&p->s1_ab, s1_band_doubles(ny, p->Nk) * sizeof(double)));
        std::vector<double> w2(5 * ny), c(3 * 5);
        for (int j = 0; j < ny; ++j) {
            const int a = std::min(std::max(j - 2, 0), ny - 5);
            fornberg(p->y.data() + a, 5, p->y[j], 2, c.data());
            for (int l = 0; l < 5; ++l) w2[5 * j + l] = c[2 * 5 + l];
        }
        CUDA_TRY(p, cudaMemcpy(p->s1_w2, w2.data(), w2.size() * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(p, s1_set_attrs(d.nx, d.nz));
        p->launches += s1_factor_launch(ny, d.nz, d.nx, d.Lx, d.Lz, p->fdw, p->s1_w2, p->fdl0, p->s1_ab, p->s1_piv,
                                        st);
        CUDA_TRY(p, cudaGetLastError());
        p->s1_ready = true;
    }
    const bool din = is_device_ptr(v_eta), dout = is_device_ptr(fields), dmean = is_device_ptr(mean_uw);
    if (!din && !p->s1_in) CUDA_TRY(p, cudaMalloc((void**)&p->s1_in, (size_t)2 * fs * sizeof(zd)));
    if (!dout && !p->s1_out) CUDA_TRY(p, cudaMalloc((void**)&p->s1_out, (size_t)4 * fs * sizeof(zd)));
    for (int s = 0; s < nsnap; ++s) {
        const zd* in = (const zd*)v_eta + (size_t)s * 2 * fs;
        if (!din) {
            CUDA_TRY(p, cudaMemcpyAsync(p->s1_in, in, (size_t)2 * fs * sizeof(zd), cudaMemcpyHostToDevice, st));
            in = p->s1_in;
        }
        CUDA_TRY(p, cudaMemcpyAsync(p->s1_mean, mean_uw + (size_t)s * 2 * ny, (size_t)2 * ny * sizeof(double),
                                    dmean ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        zd* out = dout ? (zd*)fields + (size_t)s * 4 * fs : p->s1_out;
        p->launches += s1_snapshot_launch(in, p->s1_mean, ny, d.nz, d.nx, d.Lx, d.Lz, d.nu, p->fdw, p->s1_w2, p->fdl0,
                                          p->tw_xd, p->tw_zd, p->s1_ab, p->s1_piv, p->s1_A, p->s1_B, out, st);
        CUDA_TRY(p, cudaGetLastError());
        if (!dout) {
            CUDA_TRY(p, cudaMemcpyAsync((zd*)fields + (size_t)s * 4 * fs, p->s1_out, (size_t)4 * fs * sizeof(zd),
                                        cudaMemcpyDeviceToHost, st));
            CUDA_TRY(p, cudaStreamSynchronize(st));
        }
    }
    if (!din || !dmean) CUDA_TRY(p, cudaStreamSynchronize(st));
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

// Host output: A, Phi_x, Phi_z and xi are final once the row pass of a pair
// chunk has run (the Step-3 stencils change Phi_y, phi and the residual only),
// so their rows of that chunk go to the host on a second stream while the
// later chunks and the stencils run.
static const int EARLY_TERMS[4] = {GKE_TERM_A, GKE_TERM_PHI_X, GKE_TERM_PHI_Z, GKE_TERM_XI};

static void copy_chunk(void* ctx, long long p0, long long np, cudaStream_t st)
{
    gke_plan_t p = (gke_plan_t)ctx;
    if (!p->host_terms) return;
    cudaEvent_t ev = take_event(p);
    cudaEventRecord(ev, st);
    cudaStreamWaitEvent(p->copy_st, ev, 0);
    p->chunk_ev.push_back(ev);
    const size_t row = (size_t)p->sep.nrz * p->sep.nrx * p->tsz;
    for (int t : EARLY_TERMS) {
        if (!((p->tset >> t) & 1u)) continue;
        const size_t off = ((size_t)t * p->npair + (size_t)p0) * row;
        cudaMemcpyAsync((char*)p->host_terms + off, (const char*)p->stage_terms + off, (size_t)np * row,
                        cudaMemcpyDeviceToHost, p->copy_st);
    }
}

static void terms_stage(gke_plan_t p, void* terms_dev)
{
    const gke_desc& d = p->d;
    const bool f32 = (d.precision != GKE_PREC_F64);
    // transform sizes: the grid, or the coarse grid of uniform undersampling
    const Tiles t = pick_tiles(p->nxt, p->nzt, p->csz);
    TermArgs a;
    a.fp32 = f32; a.comb64 = p->comb_is64;
    a.comb = p->comb_is64 ? (const void*)p->comb : (const void*)p->comb32;
    if (p->wedge) a.comb = p->fold;
    a.W = p->W; a.spec = p->spec; a.pair_i = p->pair_i; a.npair = p->npair; a.pair_chunk = p->pair_chunk;
    a.ny = d.ny; a.nz = p->nzt; a.nx = p->nxt;
    a.cw = t.cw_tc;
    a.rz = t.rz_tr;
    a.inv_count = 1.0 / p->snap_count; a.prof = p->prof;
    a.tw_x = f32 ? (const void*)p->ttw_xf : (const void*)p->ttw_xd;
    a.tw_z = f32 ? (const void*)p->ttw_zf : (const void*)p->ttw_zd;
    a.terms = terms_dev; a.sep = p->sep; a.st = p->st;
    a.after_chunk = copy_chunk;
    a.ctx = p;
    if (p->planes) {
        a.planes = p->pl_is64 ? (const void*)p->pl64 : (const void*)p->pl32;
        a.planes64 = p->pl_is64;
        a.npp = p->npp;
        a.Kc = p->Nk;
        a.Lx = d.Lx; a.Lz = d.Lz; a.nu = d.nu;
    }
    a.st2 = p->aux_st;
    a.W2 = p->W2;
    a.ev = p->aux_ev + 6;
    a.tmask = p->tset;
    p->launches += terms_launch(a);
}

static gke_status finalize_impl(gke_plan_t p, void* terms_dev)
{
    const gke_desc& d = p->d;
    const int ny = d.ny;
    cudaStream_t st = p->st;
    {
        StageScope sc(p, GKE_STAGE_TERMS);
        k_profiles<<<(ny + 127) / 128, 128, 0, st>>>(p->mean_sum, p->mean_count, p->stats, p->snap_count,
                                                      (long long)d.nx * d.nz, d.nu, p->wedge ? 1 : 0, p->fdw, p->fdl0, ny, p->prof);
        p->launches += 1;
        if (p->wedge) {
            // the wedge's output pairs: mirror average of the triangle's spectra
            // (full or, in the chunked mode, coarse; aliasing commutes with it)
            const int nk = p->dec ? p->nzt * (p->nxt / 2 + 1) : p->Nk;
            p->launches += mirror_fold_launch(p->comb_is64, p->comb_is64 ? (const void*)p->comb : (const void*)p->comb32,
                                              p->pair_i, p->npair, ny, nk, p->fold, st);
        }
        terms_stage(p, terms_dev);
    }
    {
        StageScope sc(p, GKE_STAGE_STENCIL);
        p->launches += stencil_launch(d.precision != GKE_PREC_F64, p->wedge ? 1 : 0, terms_dev, p->spec, p->npair,
                                      p->pair_i, ny, p->sep, d.nu, p->fdw, p->fdl0, p->prof, p->tset, st);
    }
    CUDA_TRY(p, cudaGetLastError());
    return GKE_OK;
}

// user-visible profiles [GKE_NPROF][ny] are the first GKE_NPROF rows of prof
static_assert((int)PR_U == (int)GKE_PROF_U && (int)PR_V == (int)GKE_PROF_V && (int)PR_W == (int)GKE_PROF_W &&
              (int)PR_P == (int)GKE_PROF_P && (int)PR_DU == (int)GKE_PROF_DUDY && (int)PR_EPS == (int)GKE_PROF_EPS,
              "profile order");

extern "C" gke_status gke_finalize_terms(gke_plan_t p, void* terms, double* profiles)
{
    if (!p || !terms) return p ? fail(p, GKE_ERR_ARG, "terms is NULL") : GKE_ERR_ARG;
    if (!p->have_acc || p->snap_count <= 0) return fail(p, GKE_ERR_STATE, "no snapshots accumulated");
    const bool dev_out = is_device_ptr(terms);
    const size_t tbytes = (size_t)gke_terms_bytes(p);
    void* tdev = terms;
    // pinned host output: copies overlap the remaining work (pageable memory
    // would make each early copy block the launching thread)
    const bool early = !dev_out && is_pinned_host_ptr(terms);
    if (!dev_out) {
        if (!p->stage_terms) CUDA_TRY(p, dalloc(&p->stage_terms, tbytes / sizeof(double)));
        if (early && !p->copy_st) CUDA_TRY(p, cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking));
        tdev = p->stage_terms;
        p->host_terms = early ? terms : nullptr;
    }
    gke_status s = finalize_impl(p, tdev);
    p->host_terms = nullptr;
    if (s != GKE_OK) return s;
    if (!dev_out && !early) {
        // the planes of the plan's term set
        const size_t plane = tbytes / NTERM;
        for (int t = 0; t < NTERM; ++t) {
            if (!((p->tset >> t) & 1u)) continue;
            int t1 = t;
            while (t1 + 1 < NTERM && ((p->tset >> (t1 + 1)) & 1u)) ++t1;       // runs of planes in one copy
            CUDA_TRY(p, cudaMemcpyAsync((char*)terms + t * plane, (const char*)tdev + t * plane,
                                        (size_t)(t1 - t + 1) * plane, cudaMemcpyDeviceToHost, p->st));
            t = t1;
        }
    }
    if (early) {
        // the remaining terms (Phi_y, phi, residual) after the stencils; then
        // the main stream waits for the early copies
        const size_t row = (size_t)p->sep.nrz * p->sep.nrx * p->tsz * (size_t)p->npair;
        for (int t : {GKE_TERM_PHI_Y, GKE_TERM_PHI, GKE_TERM_RESIDUAL})
            if ((p->tset >> t) & 1u) CUDA_TRY(p, cudaMemcpyAsync((char*)terms + (size_t)t * row, (const char*)tdev + (size_t)t * row, row,
                                        cudaMemcpyDeviceToHost, p->st));
        cudaEvent_t done = take_event(p);
        CUDA_TRY(p, cudaEventRecord(done, p->copy_st));
        CUDA_TRY(p, cudaStreamWaitEvent(p->st, done, 0));
        p->chunk_ev.push_back(done);
    }
    if (profiles)
        CUDA_TRY(p, cudaMemcpyAsync(profiles, p->prof, GKE_NPROF * p->d.ny * sizeof(double), cudaMemcpyDefault, p->st));
    int bad = 0;
    CUDA_TRY(p, cudaMemcpyAsync(&bad, p->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(p, cudaStreamSynchronize(p->st));
    for (cudaEvent_t e : p->chunk_ev) p->spare.push_back(e);
    p->chunk_ev.clear();
    p->finalized = true;
    if (p->d.precision == GKE_PREC_BF16X3) {
        gke_status ss = split_check(p->split, p->st, p->err);
        if (ss != GKE_OK) return ss;
    }
    if (bad) return fail(p, GKE_ERR_NONFINITE, "non-finite value in the accumulated input");
    return GKE_OK;
}

// Pinned host input of gke_compute, streamed: the k = 0 coefficients of every
// (snapshot, field, y) into k0buf on the main stream (all the Step-1 mean
// reads), then whole snapshots into stage_in on the upload stream, snapshot s
// announced by up_ev[s], so the products of the first snapshots overlap the
// copies of the later ones.
static gke_status upload_streamed(gke_plan_t p, const zd* host, int nsnap)
{
    const int ny = p->d.ny;
    const size_t per = (size_t)4 * ny * p->Nk;
    if (!p->stage_in) CUDA_TRY(p, dalloc(&p->stage_in, (size_t)p->d.max_snap * per));
    if (!p->k0buf) CUDA_TRY(p, dalloc(&p->k0buf, (size_t)p->d.max_snap * 4 * ny));
    if (!p->up_st) CUDA_TRY(p, cudaStreamCreateWithFlags(&p->up_st, cudaStreamNonBlocking));
    while ((int)p->up_ev.size() < nsnap) {
        cudaEvent_t e;
        CUDA_TRY(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->up_ev.push_back(e);
    }
    CUDA_TRY(p, cudaMemcpy2DAsync(p->k0buf, sizeof(zd), host, (size_t)p->Nk * sizeof(zd), sizeof(zd),
                                  (size_t)nsnap * 4 * ny, cudaMemcpyHostToDevice, p->st));
    // the upload stream starts after the main stream's earlier work (which may
    // still read stage_in)
    cudaEvent_t e0 = take_event(p);
    CUDA_TRY(p, cudaEventRecord(e0, p->st));
    CUDA_TRY(p, cudaStreamWaitEvent(p->up_st, e0, 0));
    p->chunk_ev.push_back(e0);
    for (int s = 0; s < nsnap; ++s) {
        CUDA_TRY(p, cudaMemcpyAsync(p->stage_in + s * per, host + s * per, per * sizeof(zd), cudaMemcpyHostToDevice,
                                    p->up_st));
        CUDA_TRY(p, cudaEventRecord(p->up_ev[s], p->up_st));
    }
    return GKE_OK;
}

extern "C" gke_status gke_compute(gke_plan_t p, const void* fields, int nsnap, void* terms, double* profiles)
{
    if (!p || !fields || !terms) return p ? fail(p, GKE_ERR_ARG, "NULL argument") : GKE_ERR_ARG;
    if (nsnap < 1 || nsnap > p->d.max_snap) return fail(p, GKE_ERR_ARG, "nsnap out of range [1, max_snap]");
    gke_status s = gke_reset(p);
    if (s != GKE_OK) return s;
    if (!is_device_ptr(fields) && is_pinned_host_ptr(fields)) {
        if ((s = upload_streamed(p, (const zd*)fields, nsnap)) != GKE_OK) return s;
        if ((s = mean_impl(p, p->k0buf, nsnap, 1)) != GKE_OK) return s;
        p->up_active = p->up_ev.data();
        s = snapshot_impl(p, p->stage_in, nsnap);
        p->up_active = nullptr;
        if (s != GKE_OK) return s;
        return gke_finalize_terms(p, terms, profiles);
    }
    const zd* f;
    if ((s = device_fields(p, fields, nsnap, &f)) != GKE_OK) return s;
    if ((s = mean_impl(p, f, nsnap)) != GKE_OK) return s;
    if ((s = snapshot_impl(p, f, nsnap)) != GKE_OK) return s;
    return gke_finalize_terms(p, terms, profiles);
}

// ------------------------------------------------------------- graph replay
// One pass as a pure device sequence (reset, Step-1 mean frozen on the device,
// the batch, Step 3), for capture into a CUDA graph.
static gke_status capture_pass(gke_plan_t p, const zd* f, int nsnap, void* terms, double* profiles)
{
    const gke_desc& d = p->d;
    const int ny = d.ny;
    cudaStream_t st = p->st;
    CUDA_TRY(p, cudaMemsetAsync(p->mean_sum, 0, 4 * ny * sizeof(double), st));
    CUDA_TRY(p, cudaMemsetAsync(p->stats, 0, NSTAT * ny * sizeof(double), st));
    CUDA_TRY(p, cudaMemsetAsync(p->nonfinite, 0, sizeof(int), st));
    if (p->dec) CUDA_TRY(p, cudaMemsetAsync(p->comb, 0, p->n_acc * sizeof(zd), st));
    gke_status s = mean_impl(p, f, nsnap);
    if (s != GKE_OK) return s;
    k_freeze_mean<<<1, 1024, 0, st>>>(p->mean_sum, p->mean_count, p->wedge ? 1 : 0, ny, p->mean);
    k_profiles<<<(ny + 127) / 128, 128, 0, st>>>(p->mean_sum, p->mean_count, p->stats, 1.0, (long long)d.nx * d.nz,
                                                  d.nu, p->wedge ? 1 : 0, p->fdw, p->fdl0, ny, p->prof);
    p->launches += 2;
    p->mean_frozen = true;
    if ((s = enqueue_snapshot(p, f, nsnap)) != GKE_OK) return s;
    if ((s = finalize_impl(p, terms)) != GKE_OK) return s;
    if (profiles)
        CUDA_TRY(p, cudaMemcpyAsync(profiles, p->prof, GKE_NPROF * ny * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return GKE_OK;
}

extern "C" gke_status gke_compute_graph(gke_plan_t p, const void* fields, int nsnap, void* terms, double* profiles)
{
    if (!p || !fields || !terms) return p ? fail(p, GKE_ERR_ARG, "NULL argument") : GKE_ERR_ARG;
    if (nsnap < 1 || nsnap > p->d.max_snap) return fail(p, GKE_ERR_ARG, "nsnap out of range [1, max_snap]");
    if (!is_device_ptr(fields) || !is_device_ptr(terms) || (profiles && !is_device_ptr(profiles)))
        return fail(p, GKE_ERR_ARG, "gke_compute_graph takes device pointers only");
    if (p->st == nullptr || p->st == cudaStreamLegacy || p->st == cudaStreamPerThread)
        return fail(p, GKE_ERR_UNSUPPORTED, "gke_compute_graph needs a plan created on a non-default stream");
    const bool same = p->graph && p->g_fields == fields && p->g_terms == terms && p->g_prof == profiles &&
                      p->g_nsnap == nsnap;
    auto fresh = [&]() {
        p->mean_count = 0.0;
        p->snap_count = 0.0;
        p->mean_frozen = p->have_acc = p->finalized = false;
        p->comb_is64 = (p->d.precision == GKE_PREC_F64) || p->dec;
        p->pl_is64 = false;
    };
    if (!same) {
        if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
        const bool timing = p->timing;
        const long long l0 = p->launches;
        p->timing = false;
        fresh();
        CUDA_TRY(p, cudaStreamSynchronize(p->st));
        cudaError_t e = cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { p->timing = timing; return fail(p, GKE_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e)); }
        const gke_status cs = capture_pass(p, (const zd*)fields, nsnap, terms, profiles);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(p->st, &g);
        p->timing = timing;
        if (cs != GKE_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return cs != GKE_OK ? cs : fail(p, GKE_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&p->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { p->graph = nullptr; return fail(p, GKE_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e)); }
        p->g_launches = p->launches - l0;
        p->launches = l0;
        p->g_fields = fields; p->g_terms = terms; p->g_prof = profiles; p->g_nsnap = nsnap;
    }
    // host state of the pass the graph runs
    fresh();
    p->mean_count = p->snap_count = nsnap;
    p->mean_frozen = p->have_acc = true;
    CUDA_TRY(p, cudaGraphLaunch(p->graph, p->st));
    p->launches += p->g_launches;
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

// ------------------------------------------------------- checkpoint files
static const int CKPT_VERSION = 5;
static_assert(sizeof(int) == 4 && sizeof(double) == 8, "checkpoint layout");

// acc_kind: 0 = per-pair term spectra comb[npair][NTERM][...], 1 = the plane
// spectra of the split plane mode [NPLANE][npair / 4][Nk][4]
struct CkptHeader {
    char magic[8];
    int version, nx, nz, ny, precision, have_acc, pair_domain, nzt, nxt, term_set, acc_kind, reserved;
    double mean_count, snap_count, Lx, Lz, nu;
};

static_assert(sizeof(CkptHeader) == 96, "checkpoint header layout");

// largest difference between two mean profiles that still counts as the same
// mean (rounding of sums taken in another order)
static bool same_mean(const std::vector<double>& a, const std::vector<double>& b)
{
    double scale = 0.0, diff = 0.0;
    for (size_t i = 0; i < a.size(); ++i) {
        scale = std::max(scale, std::max(std::fabs(a[i]), std::fabs(b[i])));
        diff = std::max(diff, std::fabs(a[i] - b[i]));
    }
    return diff <= 1e-12 * std::max(scale, 1e-300);
}

static gke_status ckpt_io(gke_plan_t p, const char* path, int mode)   // 0 save, 1 restore, 2 merge
{
    if (!p || !path) return p ? fail(p, GKE_ERR_ARG, "path is NULL") : GKE_ERR_ARG;
    const int ny = p->d.ny;
    const size_t n_mean = 4 * ny, n_stat = (size_t)NSTAT * ny;
    const size_t n_comb = p->n_acc;
    const int acc_kind = p->planes ? 1 : p->dec ? 2 : 0;
    // the stored sums are FP64; a split plan holding one batch in FP32 promotes first
    if (p->planes) {
        if (p->have_acc && !p->pl_is64) {
            if (!p->pl64) CUDA_TRY(p, dalloc(&p->pl64, n_comb));
            planes_accum_launch(p->pl32, (long long)p->Nk * p->npp, (1u << NPLANE) - 1u, 0, p->pl64, p->st);
            p->pl_is64 = true;
        }
        if (mode != 0 && !p->pl64) CUDA_TRY(p, dalloc(&p->pl64, n_comb));
    } else {
        if (p->have_acc && !p->comb_is64) {
            if (!p->comb) CUDA_TRY(p, dalloc(&p->comb, n_comb));
            promote_launch(p->comb32, (long long)n_comb, p->comb, p->st);
            p->comb_is64 = true;
        }
        if (mode != 0 && !p->comb) CUDA_TRY(p, dalloc(&p->comb, n_comb));
    }
    zd* accp = p->planes ? p->pl64 : p->comb;
    CUDA_TRY(p, cudaStreamSynchronize(p->st));
    // the mean the accumulated spectra were taken about (frozen by the first batch)
    std::vector<double> frozen(n_mean, 0.0);
    if (p->have_acc) CUDA_TRY(p, cudaMemcpy(frozen.data(), p->mean, n_mean * 8, cudaMemcpyDeviceToHost));
    if (mode == 0) {
        FILE* fp = fopen(path, "wb");
        if (!fp) return fail(p, GKE_ERR_IO, std::string("cannot open for writing: ") + path);
        CkptHeader h{};
        memcpy(h.magic, "GKECKPT", 8);
        h.version = CKPT_VERSION; h.nx = p->d.nx; h.nz = p->d.nz; h.ny = ny; h.precision = p->d.precision;
        h.have_acc = p->have_acc; h.mean_count = p->mean_count; h.snap_count = p->snap_count;
        h.Lx = p->d.Lx; h.Lz = p->d.Lz; h.nu = p->d.nu;
        h.pair_domain = p->d.pair_domain;
        h.nzt = p->dec ? p->nzt : 0;
        h.nxt = p->dec ? p->nxt : 0;
        h.term_set = (int)p->tset;
        h.acc_kind = acc_kind;
        bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
        std::vector<char> buf;
        auto put = [&](const void* dptr, size_t bytes) {
            buf.resize(bytes);
            if (cudaMemcpy(buf.data(), dptr, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
            return fwrite(buf.data(), 1, bytes, fp) == bytes;
        };
        ok = ok && put(p->mean_sum, n_mean * 8) && put(p->stats, n_stat * 8);
        if (p->have_acc) {
            ok = ok && fwrite(frozen.data(), 8, n_mean, fp) == n_mean;
            ok = ok && put(accp, n_comb * 16);
        }
        ok = (fclose(fp) == 0) && ok;
        return ok ? GKE_OK : fail(p, GKE_ERR_IO, std::string("write failed: ") + path);
    }
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(p, GKE_ERR_IO, std::string("cannot open for reading: ") + path);
    CkptHeader h{};
    if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, "GKECKPT", 8) != 0 || h.version != CKPT_VERSION) {
        fclose(fp);
        return fail(p, GKE_ERR_IO, "not a GKE checkpoint of this version");
    }
    if (h.nx != p->d.nx || h.nz != p->d.nz || h.ny != ny || h.Lx != p->d.Lx || h.Lz != p->d.Lz || h.nu != p->d.nu ||
        h.pair_domain != p->d.pair_domain || h.nzt != (p->dec ? p->nzt : 0) || h.nxt != (p->dec ? p->nxt : 0) ||
        h.term_set != (int)p->tset) {
        fclose(fp);
        return fail(p, GKE_ERR_ARG, "checkpoint grid, domain or term set does not match the plan");
    }
    if (h.have_acc && h.acc_kind != acc_kind) {
        fclose(fp);
        return fail(p, GKE_ERR_ARG, "checkpoint accumulator layout does not match the plan (per-pair term spectra, "
                                    "plane spectra of the split path, or coarse spectra of the chunked mode)");
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
    // the file's frozen mean follows its one-point sums; read the sums into
    // host memory first so a refused merge leaves the plan unchanged
    std::vector<double> f_mean_sum(n_mean), f_stats(n_stat), f_frozen(n_mean);
    ok = fread(f_mean_sum.data(), 8, n_mean, fp) == n_mean && fread(f_stats.data(), 8, n_stat, fp) == n_stat;
    if (ok && h.have_acc) ok = fread(f_frozen.data(), 8, n_mean, fp) == n_mean;
    if (!ok) { fclose(fp); return fail(p, GKE_ERR_IO, std::string("read failed or truncated: ") + path); }
    const bool add = (mode == 2);
    if (add && p->have_acc && h.have_acc && !same_mean(frozen, f_frozen)) {
        fclose(fp);
        return fail(p, GKE_ERR_ARG, "checkpoint spectra were taken about another Step-1 mean: jobs to be merged "
                                    "must share the mean (gke_set_mean, or gke_accumulate_mean over the same "
                                    "snapshots)");
    }
    {
        std::vector<double> cur(n_mean), curs(n_stat);
        if (add) {
            CUDA_TRY(p, cudaMemcpy(cur.data(), p->mean_sum, n_mean * 8, cudaMemcpyDeviceToHost));
            CUDA_TRY(p, cudaMemcpy(curs.data(), p->stats, n_stat * 8, cudaMemcpyDeviceToHost));
        }
        for (size_t i = 0; i < n_mean; ++i) cur[i] = (add ? cur[i] : 0.0) + f_mean_sum[i];
        for (size_t i = 0; i < n_stat; ++i) curs[i] = (add ? curs[i] : 0.0) + f_stats[i];
        CUDA_TRY(p, cudaMemcpy(p->mean_sum, cur.data(), n_mean * 8, cudaMemcpyHostToDevice));
        CUDA_TRY(p, cudaMemcpy(p->stats, curs.data(), n_stat * 8, cudaMemcpyHostToDevice));
    }
    if (h.have_acc) {
        const bool add_acc = add && p->have_acc;
        get(accp, n_comb * 16, false, add_acc);
    }
    fclose(fp);
    if (!ok) return fail(p, GKE_ERR_IO, std::string("read failed or truncated: ") + path);
    if (h.have_acc) {
        if (p->planes) p->pl_is64 = true;
        else p->comb_is64 = true;
    }
    const bool had_acc = p->have_acc;
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
        // the mean the accumulated spectra were taken about: the plan's own, or
        // the file's when the plan had no samples yet
        const std::vector<double>& m = (add && had_acc) ? frozen : f_frozen;
        CUDA_TRY(p, cudaMemcpy(p->mean, m.data(), m.size() * 8, cudaMemcpyHostToDevice));
        k_profiles<<<(ny + 127) / 128, 128, 0, p->st>>>(p->mean_sum, p->mean_count, p->stats, 1.0,
                                                         (long long)p->d.nx * p->d.nz, p->d.nu, p->wedge ? 1 : 0,
                                                         p->fdw, p->fdl0, ny, p->prof);
        CUDA_TRY(p, cudaStreamSynchronize(p->st));
        p->mean_frozen = true;
    }
    p->finalized = false;
    return GKE_OK;
}

extern "C" gke_status gke_checkpoint(gke_plan_t p, const char* path) { return ckpt_io(p, path, 0); }
extern "C" gke_status gke_restore(gke_plan_t p, const char* path) { return ckpt_io(p, path, 1); }
extern "C" gke_status gke_merge(gke_plan_t p, const char* path) { return ckpt_io(p, path, 2); }
