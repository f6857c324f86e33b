// gke_split.cu -- split-precision correlator on the 5th-generation tensor cores.
//
// The per-wavenumber contractions of the Parseval step (Sec. 3.1, Eq. 8-9),
//   S(y, y') = sum_t sum_s conj(A_t[s][y]) B_t[s][y'],
// written as real products (Re S = ar br + ai bi, Im S = ar bi - ai br) with
// every real operand split into three BF16 slices x = x0 + x1 + x2 (each the
// BF16 rounding of what the previous ones leave; BF16 has the FP32 exponent
// range, so every slice is relative to its own value and no scaling is
// needed).  The six slice products with i + j <= 2 keep ~24 significant bits:
//   x y ~ x0 y0 + x0 y1 + x1 y0 + x0 y2 + x1 y1 + x2 y0,
// accumulated in FP32 in tensor memory and written as the batch's FP32
// contraction raw[job][k][y][y'] (k_combine then adds it, in FP64, to the
// per-pair term spectra).
// FP32 accumulation rounds against the running sum, so the small cross-slice
// products of all terms go first and the large x0 y0 products last: an output
// then sees 2 T G large additions (T terms, G snapshot groups) instead of 12 T G.
//
// Tensor-core mapping (one work item = one wavenumber k, one contraction,
// one 128 x 128 tile of (y, y')): D[128 x 256] in TMEM, columns 0..127 = Re,
// 128..255 = Im.  Per term, snapshot group of 16 and slice pair (i, j):
//   mma(A = ar_i, B = [br_j | bi_j], N = 256)       -> Re += ar br, Im += ar bi
//   mma(A = ai_i, B = bi_j, N = 128) into Re         -> Re += ai bi
//   mma(A = -ai_i, B = br_j, N = 128) into Im        -> Im -= ai br
// (M = 128, K = 16, BF16 in, FP32 accumulate; the sign by the negate-A bit
// of the instruction descriptor).  The B block holds the rows br, bi back to
// back, so every B view is a window of it.  Operands are written by
// k_split_prep_* in the canonical K-major
// no-swizzle layout (8 x 16-byte core matrices; K-adjacent core matrices LBO
// bytes apart, M/N-adjacent ones SBO = 128 bytes apart) and copied to shared
// memory by the bulk-copy engine (cp.async.bulk, mbarrier transaction count).
// Wall-normal sizes ny = 128 m + 1 (Chebyshev-Gauss-Lobatto grids) leave one
// row and one column outside the tiles; k_corr_edge does those in FP32 on the
// CUDA cores.
#include <cuda_bf16.h>

#include <algorithm>

#include "gke_split.h"
#include "gke_kernels.h"

namespace gke {

typedef __nv_bfloat16 bf16;

constexpr int TM = 128;                 // tile rows (y) = tile cols (y')
constexpr int KS = 16;                  // snapshots per group = one MMA K step
constexpr int A_BLK = TM * KS;          // bf16 per A block (128 rows x 16)
constexpr int B_BLK = 2 * TM * KS;      // bf16 per B block (br | bi rows x 16)
constexpr int A_STAGE = 6 * A_BLK;      // slices x parts (re, im), slice-major
constexpr int B_STAGE = 3 * B_BLK;      // slices
constexpr int SM_A = A_STAGE * 2;       // 24576 bytes
constexpr int SM_B = B_STAGE * 2;       // 24576 bytes
constexpr int NFB = 4;                  // B operand slots per wavenumber: u, v, w, 2 U'(y) v
constexpr int A_LBO = (TM / 8) * 128;       // 2048: K-adjacent core matrices in an A block
constexpr int B_LBO = (2 * TM / 8) * 128;   // 4096: K-adjacent core matrices in a B block
constexpr int CM_SBO = 128;                 // M/N-adjacent core matrices

// instruction descriptor, kind::f16: D = F32 (bits 4-5), A = B = BF16 (7-9, 10-12),
// K-major A and B (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t IDESC_N128 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                                ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t NEG_A = 1u << 13;       // negate-A bit of the instruction descriptor

// one contraction: sum over its terms t of sign_t conj(A_fa[t]) B_fb[t]; bit t
// of neg marks a term with sign -1 (the MMA's negate-A bit)
struct TcJob { int nterm; int fa[5]; int fb[5]; unsigned neg; };
__constant__ TcJob c_tcjobs[NJSQ + 1];
__constant__ TcJob c_tcplanes[NPLANE];
// planes of an off-diagonal tile pair (y in tile mt < nt, y' in tile nt): as
// c_tcplanes, except that xi takes B = 2 U'(y') v (slot 3), so that the
// partner-free form below needs no per-row factor
__constant__ TcJob c_tcoff[NPLANE];

// cross-slice pairs (i, j), 0 < i + j <= 2; the pair (0, 0) goes last
__constant__ int c_pi[5] = {1, 0, 2, 1, 0};
__constant__ int c_pj[5] = {1, 2, 0, 0, 1};

// Packed K (one snapshot group of ns <= 5): the six slice products of a term
// in three MMA K steps instead of six zero-padded ones, one step per order of
// magnitude so that an MMA never sums products of different sizes: step 0
// the slice pairs (1, 1), (0, 2), (2, 0) (about 2^-16 of x0 y0), step 1
// (1, 0), (0, 1) (2^-8), step 2 (0, 0).  Position c of step ks holds slice
// pair c / ns of the step for snapshot c mod ns.  The K steps take the places
// of the slices in the operand blocks (step ks at 2 ks A_BLK elements of an A
// block and ks B_BLK = 2 ks A_BLK of a B block), so the copies and descriptors
// keep their layout; as in the unpacked order, steps 0 and 1 of every term
// go first (pass 0) and step 2 last (pass 1).
constexpr int PK_MAX_NS = 5, PK_STEPS = 3;
__device__ __forceinline__ int pk_pairs(int ks) { return 3 - ks; }      // slice pairs in step ks
// slices (i of A, j of B) of pair sp of step ks
__device__ __forceinline__ int pk_i(int ks, int sp) { return ks == 0 ? (sp == 0 ? 1 : sp == 1 ? 0 : 2) : ks == 1 ? (sp == 0 ? 1 : 0) : 0; }
__device__ __forceinline__ int pk_j(int ks, int sp) { return ks == 0 ? (sp == 0 ? 1 : sp == 1 ? 2 : 0) : ks == 1 ? (sp == 0 ? 0 : 1) : 0; }

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, int n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait: false after ~2^22 polls with back-off (about a second)
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_try(b, parity)) return true;
        if (it > 32) __nanosleep(200);
    }
    return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
// bounded wait that also gives up as soon as another role of the CTA has
// raised the abort flag
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* b, uint32_t parity, volatile int* abort) {
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_try(b, parity)) return true;
        if (*abort) return false;
        if (it > 32) __nanosleep(200);
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(b)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
// SBO >> 4 (32-45), version 1 (46-47), no swizzle (61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((su32(p) & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t dtm, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(dtm), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------ operand prep
// element (row r, k) of a core-matrix tile whose K-adjacent core matrices are
// `rows/8` cores apart: ((k/8) * rows/8 + r/8) * 64 + (r%8) * 8 + k%8
__device__ __forceinline__ int cm_index(int r, int kk, int rows) {
    return (((kk >> 3) * (rows >> 3) + (r >> 3)) << 6) + ((r & 7) << 3) + (kk & 7);
}

__device__ __forceinline__ void split3(float x, bf16& s0, bf16& s1, bf16& s2) {
    s0 = __float2bfloat16_rn(x);
    float r1 = x - __bfloat162float(s0);
    s1 = __float2bfloat16_rn(r1);
    float r2 = r1 - __bfloat162float(s1);
    s2 = __float2bfloat16_rn(r2);
}

// Aop[k][f][g][mt][slice * 2 + part][A_BLK] (the operands of uu .. vw carry the
// factor 2 of the expansion already); rows >= cov and snapshots >= ns are zero.  Thread
// = one row x 8 snapshots: the 8 values of a core-matrix row are contiguous,
// so each slice goes out as one 16-byte store.
struct alignas(16) bf16x8 { bf16 v[8]; };

__global__ void k_split_prep_A(const zf* __restrict__ Xop, int ns, int ny, int Nk, int k0, int G, int MT, int cov,
                               float pscale, int nks, bf16* __restrict__ Aop)
{
    long long b = blockIdx.x;
    const int mt = (int)(b % MT); b /= MT;
    const int g = (int)(b % G); b /= G;
    const int f = (int)(b % NFIELD);
    const int k = (int)(b / NFIELD);
    bf16* dst = Aop + ((((long long)k * NFIELD + f) * G + g) * MT + mt) * (long long)A_STAGE;
    const int r = threadIdx.x % TM, kc = threadIdx.x / TM;          // blockDim = 2 TM
    const int y = mt * TM + r;
    if (nks) {
        // packed K: the row's ns values split once, then placed by step
        bf16 sr[PK_MAX_NS][3], si[PK_MAX_NS][3];
        for (int s = 0; s < ns; ++s) {
            zf v = mk(0.f, 0.f);
            if (y < cov) v = Xop[(((long long)f * Nk + k0 + k) * ns + s) * ny + y];
            if (f == F_P) v = pscale * v;                      // a power of two: exact
            split3(v.x, sr[s][0], sr[s][1], sr[s][2]);
            split3(v.y, si[s][0], si[s][1], si[s][2]);
        }
        const int idx = cm_index(r, kc * 8, TM);
        const bf16 z = __float2bfloat16_rn(0.f);
        for (int ks = 0; ks < PK_STEPS; ++ks) {
            bf16x8 ore, oim;
            #pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int c = kc * 8 + e, sp = c / ns, s = c - sp * ns;
                const bool live = sp < pk_pairs(ks);
                const int sl = live ? pk_i(ks, sp) : 0;
                ore.v[e] = live ? sr[s][sl] : z;
                oim.v[e] = live ? si[s][sl] : z;
            }
            *(bf16x8*)(dst + (2 * ks) * A_BLK + idx) = ore;
            *(bf16x8*)(dst + (2 * ks + 1) * A_BLK + idx) = oim;
        }
        return;
    }
    bf16x8 o[6];
    #pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int s = g * KS + kc * 8 + e;
        zf v = mk(0.f, 0.f);
        if (y < cov && s < ns) v = Xop[(((long long)f * Nk + k0 + k) * ns + s) * ny + y];
        if (f == F_P) v = pscale * v;                      // a power of two: exact
        split3(v.x, o[0].v[e], o[2].v[e], o[4].v[e]);      // slices of the real part
        split3(v.y, o[1].v[e], o[3].v[e], o[5].v[e]);      // slices of the imaginary part
    }
    const int idx = cm_index(r, kc * 8, TM);
    #pragma unroll
    for (int q = 0; q < 6; ++q) *(bf16x8*)(dst + q * A_BLK + idx) = o[q];
}

// Bop[k][NFB][g][nt][slice][B_BLK], slots fb = u, v, w and (nfb = 4) the
// product 2 U'(y) v in FP32; rows br | bi
__global__ void k_split_prep_B(const zf* __restrict__ Xop, int ns, int ny, int Nk, int k0, int G, int MT, int cov,
                               int nfb, const double* __restrict__ prof, int nks, bf16* __restrict__ Bop)
{
    long long b = blockIdx.x;
    const int nt = (int)(b % MT); b /= MT;
    const int g = (int)(b % G); b /= G;
    const int fb = (int)(b % nfb);
    const int k = (int)(b / nfb);
    bf16* dst = Bop + ((((long long)k * NFB + fb) * G + g) * MT + nt) * (long long)B_STAGE;
    const int r = threadIdx.x % TM, kc = threadIdx.x / TM;          // blockDim = 2 TM
    const int y = nt * TM + r;
    const int src = fb == 3 ? F_V : fb;
    const float sc = (fb == 3 && y < ny) ? 2.f * (float)prof[PR_DU * ny + y] : 1.f;
    if (nks) {
        // packed K (see k_split_prep_A): slice pk_j of B
        bf16 sr[PK_MAX_NS][3], si[PK_MAX_NS][3];
        for (int s = 0; s < ns; ++s) {
            zf v = mk(0.f, 0.f);
            if (y < cov) v = Xop[(((long long)src * Nk + k0 + k) * ns + s) * ny + y];
            if (fb == 3) v = mk(sc * v.x, sc * v.y);
            split3(v.x, sr[s][0], sr[s][1], sr[s][2]);
            split3(v.y, si[s][0], si[s][1], si[s][2]);
        }
        const bf16 z = __float2bfloat16_rn(0.f);
        for (int ks = 0; ks < PK_STEPS; ++ks) {
            bf16x8 obr, obi;
            #pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int c = kc * 8 + e, sp = c / ns, s = c - sp * ns;
                const bool live = sp < pk_pairs(ks);
                const int sl = live ? pk_j(ks, sp) : 0;
                obr.v[e] = live ? sr[s][sl] : z;
                obi.v[e] = live ? si[s][sl] : z;
            }
            bf16* d = dst + ks * B_BLK;
            *(bf16x8*)(d + cm_index(r, kc * 8, 2 * TM)) = obr;
            *(bf16x8*)(d + cm_index(TM + r, kc * 8, 2 * TM)) = obi;
        }
        return;
    }
    bf16x8 br[3], bi[3];
    #pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int s = g * KS + kc * 8 + e;
        zf v = mk(0.f, 0.f);
        if (y < cov && s < ns) v = Xop[(((long long)src * Nk + k0 + k) * ns + s) * ny + y];
        if (fb == 3) v = mk(sc * v.x, sc * v.y);
        split3(v.x, br[0].v[e], br[1].v[e], br[2].v[e]);
        split3(v.y, bi[0].v[e], bi[1].v[e], bi[2].v[e]);
    }
    #pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
        bf16* d = dst + sl * B_BLK;
        *(bf16x8*)(d + cm_index(r, kc * 8, 2 * TM)) = br[sl];
        *(bf16x8*)(d + cm_index(TM + r, kc * 8, 2 * TM)) = bi[sl];
    }
}

// ------------------------------------------------------ tensor-core kernel
// the contractions one launch runs (a term mask may leave some out): the
// square ones, 3 bits each in sq (nsq of them), and, if d, the Hermitian D
struct TcSel { int nsq; unsigned sq; int d; };

__host__ __device__ __forceinline__ int sel_tiles(const TcSel& s, int MT)
{
    return s.nsq * MT * MT + (s.d ? MT * (MT + 1) / 2 : 0);
}

__device__ __forceinline__ void decode_tile(int jt, int MT, const TcSel& sel, int& job, int& mt, int& nt)
{
    const int sq = MT * MT;
    if (jt < sel.nsq * sq) {
        const int js = jt / sq;
        job = (int)((sel.sq >> (3 * js)) & 7u);
        int r = jt - js * sq;
        mt = r / MT;
        nt = r - mt * MT;
    } else {
        job = NJSQ;
        int r = jt - sel.nsq * sq;
        mt = 0;
        while (r >= MT - mt) { r -= MT - mt; ++mt; }
        nt = mt + r;
    }
}

// What one launch of the tensor-core kernel runs and where it writes.
//   raw mode (planes == 0): items (wavenumber, contraction, 128 x 128 tile),
//     the tile written as FP32 contractions raw[job][yb][yb'][k][8][8];
//   plane mode (planes != 0, one 128-row tile, cov <= 128): items
//     (wavenumber, plane), the plane's term spectrum of every pair
//     y <= y' < cov written to out[plane][k][pair] (FP32, npp >= npair pairs
//     per row).
struct TcArgs {
    const bf16* Aop; const bf16* Bop;
    int Kc, G, MT, ny, cov;
    long long nitems;
    TcSel sel; zf* raw;                       // raw mode
    unsigned planes; int npl; long long npp;  // plane mode: selected planes, their count, padded pair count
    int ntp;                                  // plane mode: tile pairs (mt <= nt) per wavenumber
    int nks;                                  // packed K steps (one snapshot group of <= 5), else 0
    zf* out; const double* prof;
    int* err;
};

// ------------------------------------------------ tensor-core kernel
// One CTA per SM walks the work items blockIdx.x, blockIdx.x + gridDim.x, ...
// Roles:
//   warp 0 (one lane): bulk copies of the operand blocks into a ring of NST
//     shared-memory stages (full[s] completes when a stage's bytes land);
//   warp 1 (one lane): the MMAs of an item into one of two 256-column TMEM
//     accumulators, each stage released by a commit to empty[s], the
//     finished accumulator announced by a commit to acc_full[b];
//   warps 2-5: the epilogue of an item (TMEM -> registers -> shared memory ->
//     global memory), then acc_empty[b] for the MMA warp.
// So the copies, the tensor cores and the output writes of successive items
// overlap.  Every wait is bounded; a timed-out wait raises the CTA's abort
// flag (all roles leave their loops) and the device error flag, and the copies
// and MMAs in flight are drained before the shared memory and TMEM go away.
//
// Plane-mode epilogue.  With X the accumulator (X(y, y') in TMEM lane y) and
// X^H(y, y') = conj X(y', y), the planes of one wavenumber are (Sec. 3.1,
// Eq. 7 grouped by term; the factor 2 of the expansion rides on the product
// operands):
//   A     = -2 D                          D  = sum_i conj(u_i) u_i
//   S4    = Gx - Gx^H                     Gx = conj(q) u + 2 sum_i conj(u u_i) u_i
//   Phi_y = Gy - Gy^H                     Gy = conj(q) v + 2 sum_i conj(v u_i) u_i
//   S6    = Gz - Gz^H                     Gz = conj(q) w + 2 sum_i conj(w u_i) u_i
//   phi   = (H + H^H) / 2                 H  = conj(q) v - 2 sum_i conj(v u_i) u_i - 4 conj(p) v
//   xi    = 2 U'(y') E + 2 U'(y) E^H      E  = conj(u) v
// The partner values X(y', y) come through shared memory in 32 x 32 blocks.
// Warp q holds the rows [32 q, 32 q + 32) and lays out its blocks (q, c),
// c <= q (the lower triangle of the tile, in order c = 0, 1, ..); it then
// forms its output blocks (q, b), b >= q, each from its own TMEM block and
// the block (b, q) that warp b laid out, announced by a named barrier of the
// two warps.  With these orders every warp does five block steps per item.
// A consumed block holds the warp's outputs next, so each row of 32 pairs
// leaves as one contiguous 256-byte store.  Blocks are swizzled (element
// (r, c) of a block at r * 32 + ((c + r) mod 32)), so row and column
// accesses of a half-warp hit 16 distinct bank pairs.
constexpr int NST = 3;                                  // operand stages
constexpr int EPI_WARPS = 4;
constexpr int TCP_THREADS = 64 + 32 * EPI_WARPS;
constexpr int SMP_STAGE = SM_A + SM_B;                  // 49152 bytes
constexpr int SMP_EPI = NST * SMP_STAGE;
constexpr int EPI_BLOCKS = 10;                          // lower-triangle 32 x 32 blocks of a tile
constexpr int EPI_BYTES = EPI_BLOCKS * 32 * 32 * 8;     // plane mode; raw mode uses 4 x 32 x 33 x 8
constexpr int SMP_DUP = SMP_EPI + EPI_BYTES;            // 2 U'(y) for the xi plane
constexpr int DUP_ROWS = 4 * TM;                        // rows of s_dup: plane mode covers up to 4 tiles
constexpr int SMP_BAR = SMP_DUP + DUP_ROWS * 4;
constexpr int SMP_TOTAL = SMP_BAR + 256;
constexpr uint32_t TMEM_COLS_P = 512;
static_assert(EPI_BYTES >= EPI_WARPS * 32 * 33 * 8, "raw-mode staging fits");
static_assert(SMP_TOTAL <= 232448, "shared memory of one CTA");

struct TcPipeBars {
    uint64_t full[NST], empty[NST], acc_full[2], acc_empty[2], drain;
    uint64_t bfull, bempty;                             // resident B blocks (MODE 2)
    uint32_t tmem;
    int abort;
    int eok;                                            // epilogue: the accumulator is ready
};

// named barrier of the four epilogue warps
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// named barriers 2..7 of the epilogue warp pairs (b, c), b > c: warp b
// arrives once block (b, c) is laid out, warp c waits before reading it
__device__ __forceinline__ int pair_bar(int b, int c) { return 2 + b * (b - 1) / 2 + c; }
__device__ __forceinline__ void bar_arrive64(int id) { asm volatile("bar.arrive %0, 64;" ::"r"(id) : "memory"); }
__device__ __forceinline__ void bar_sync64(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }
// slot of the lower-triangle block (b, c), c <= b; swizzled element offset
__device__ __forceinline__ int tri_slot(int b, int c) { return b * (b + 1) / 2 + c; }
__device__ __forceinline__ int swz(int r, int c) { return r * 32 + ((c + r) & 31); }

// Work of one launch, item by item (item it = blockIdx.x, blockIdx.x +
// gridDim.x, ...).  MODE 0: raw contractions, item = (wavenumber, contraction,
// tile); MODE 1: planes, item = (wavenumber, plane); MODE 2: planes, item =
// one wavenumber with all its planes in sequence ("units"), the B blocks of u,
// v, w (one snapshot group) resident in shared memory for the whole item and
// only the A blocks streamed through the stage ring.
template <int MODE> struct Units {
    int k, n, mt, nt, j0;
    unsigned planes;
    // contraction (MODE 0) or plane of unit un
    __device__ __forceinline__ int job(int un) const { return MODE == 2 ? nth_bit(planes, un) : j0; }
};
template <int MODE>
__device__ __forceinline__ Units<MODE> item_units(const TcArgs& a, int njt, long long it)
{
    Units<MODE> u;
    u.planes = a.planes;
    if (MODE == 2) {
        u.k = (int)it;
        u.n = a.npl;
        u.j0 = 0;
        u.mt = u.nt = 0;
    } else if (MODE == 1) {
        // (wavenumber, tile pair mt <= nt of the upper triangle, plane)
        const long long per_k = (long long)a.ntp * a.npl;
        u.k = (int)(it / per_k);
        const int r = (int)(it - (long long)u.k * per_k);
        u.n = 1;
        u.j0 = nth_bit(a.planes, r % a.npl);
        int tp = r / a.npl, mt = 0;
        while (tp >= a.MT - mt) { tp -= a.MT - mt; ++mt; }
        u.mt = mt;
        u.nt = mt + tp;
    } else {
        u.k = (int)(it / njt);
        u.n = 1;
        decode_tile((int)(it % njt), a.MT, a.sel, u.j0, u.mt, u.nt);
    }
    return u;
}

template <int MODE>
__device__ __forceinline__ const TcJob& job_desc(int job) { return MODE ? c_tcplanes[job] : c_tcjobs[job]; }

// Off-diagonal tile pairs of plane mode (y in tile mt < nt, every y' > y):
// a plane al X + be X^H is one accumulator without a transposition,
//   al sum_t conj(A_t(y)) B_t(y') + be sum_t conj(B_t(y)) A_t(y')
// (X^H(y, y') = conj X(y', y)), so after the jd.nterm terms X the same terms
// run "swapped": the A role takes B_t in its B-operand layout at tile mt, the
// B role A_t in its A-operand layout at tile nt (be = -1 for S4, Phi_y, S6:
// the negate bit flips; +1 for phi and xi; A has no partner terms).
__device__ __forceinline__ int off_terms(const TcJob& jd, int job) { return jd.nterm * (job == PL_A ? 1 : 2); }
__device__ __forceinline__ bool off_flip(int job) { return job == PL_S4 || job == PL_PHIY || job == PL_S6; }

// shared-memory offsets of stage st: its A block and (MODE 0, 1) its B block;
// MODE 2 keeps the three B blocks of the item at offset 0
constexpr int SMP_BRES = 3 * SM_B;                      // resident B blocks (MODE 2)
static_assert(SMP_BRES + NST * SM_A <= NST * SMP_STAGE, "resident B and the A ring fit the stage area");
template <int MODE> __device__ __forceinline__ int stage_a(int st) { return MODE == 2 ? SMP_BRES + st * SM_A : st * SMP_STAGE; }

template <int MODE>
__global__ void __launch_bounds__(TCP_THREADS, 1)
k_corr_tc_pipe(const TcArgs a)
{
    constexpr bool PLANES = MODE != 0;
    extern __shared__ __align__(1024) uint8_t smem[];
    TcPipeBars* bars = (TcPipeBars*)(smem + SMP_BAR);
    volatile int* abort = &bars->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int njt = PLANES ? a.npl : sel_tiles(a.sel, a.MT);
    const int G = a.G, MT = a.MT;
    if (threadIdx.x == 0) {
        for (int st = 0; st < NST; ++st) {
            mbar_init(&bars->full[st], 1);
            mbar_init(&bars->empty[st], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], EPI_WARPS);
        }
        mbar_init(&bars->drain, 1);
        mbar_init(&bars->bfull, 1);
        mbar_init(&bars->bempty, 1);
        bars->abort = (*(volatile int*)a.err != 0) ? 1 : 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (PLANES) {
        float* s_dup = (float*)(smem + SMP_DUP);
        for (int i = threadIdx.x; i < DUP_ROWS; i += blockDim.x)
            s_dup[i] = i < a.ny ? 2.f * (float)a.prof[PR_DU * a.ny + i] : 0.f;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&bars->tmem)),
                     "r"(TMEM_COLS_P) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tmem;
    auto fail = [&]() { *abort = 1; atomicExch(a.err, 1); };

    if (warp == 0) {
        if (lane == 0) {
            int st = 0;
            uint32_t ph = 0, bph = 0;
            int issued = 0, b_issued = 0;
            for (long long it = blockIdx.x; it < a.nitems && !*abort; it += gridDim.x) {
                const Units<MODE> u = item_units<MODE>(a, njt, it);
                const int k = u.k;
                // MODE 2: the item's B blocks replace the previous item's once
                // its MMAs are done; the first NST A stages of the item go
                // out before that wait, so the ring does not drain between items
                bool b_done = MODE != 2;
                int sidx = 0;
                auto load_b = [&]() -> bool {
                    if (!mbar_wait_ab(&bars->bempty, bph ^ 1, abort)) return false;
                    const uint32_t bres = a.nks ? a.nks * B_BLK * 2 : SM_B;
                    mbar_expect_tx(&bars->bfull, 3 * bres);
                    for (int fb = 0; fb < 3; ++fb)
                        bulk_g2s(smem + fb * SM_B, a.Bop + ((long long)k * NFB + fb) * G * MT * (long long)B_STAGE, bres,
                                 &bars->bfull);
                    ++b_issued;
                    bph ^= 1;
                    b_done = true;
                    return true;
                };
                for (int un = 0; un < u.n; ++un) {
                    const int job = u.job(un);
                    const bool off = MODE == 1 && u.mt != u.nt;
                    const TcJob& jd = off ? c_tcoff[job] : job_desc<MODE>(job);
                    const int nterm = off ? off_terms(jd, job) : jd.nterm;
                    // pass 0: the cross slices (packed: K steps 0 and 1), pass 1: (0, 0)
                    for (int pass = 0; pass < 2; ++pass)
                        for (int tt = 0; tt < nterm; ++tt)
                            for (int g = 0; g < G; ++g) {
                                if (!mbar_wait_ab(&bars->empty[st], ph ^ 1, abort)) { fail(); goto producer_done; }
                                const bool sw = tt >= jd.nterm;
                                const int t = sw ? tt - jd.nterm : tt;
                                const uint32_t ba = pass ? 2 * A_BLK * 2 : a.nks ? 4 * A_BLK * 2 : SM_A;
                                const uint32_t bb = pass ? B_BLK * 2 : a.nks ? 2 * B_BLK * 2 : SM_B;
                                // packed pass 1 copies K step 2 (offset 4 A_BLK = 2 B_BLK in either layout)
                                const long long po = (a.nks && pass) ? 4LL * A_BLK : 0;
                                uint8_t* sa = smem + stage_a<MODE>(st);
                                mbar_expect_tx(&bars->full[st], MODE == 2 ? ba : ba + bb);
                                const bf16* asrc = a.Aop + ((((long long)k * NFIELD + jd.fa[t]) * G + g) * MT +
                                                            (sw ? u.nt : u.mt)) * (long long)A_STAGE;
                                const bf16* bsrc = a.Bop + ((((long long)k * NFB + jd.fb[t]) * G + g) * MT +
                                                            (sw ? u.mt : u.nt)) * (long long)B_STAGE;
                                // swapped terms: the B operand's block in the A slot and vice versa
                                bulk_g2s(sa, (sw ? bsrc : asrc) + po, ba, &bars->full[st]);
                                if (MODE != 2) bulk_g2s(sa + SM_A, (sw ? asrc : bsrc) + po, bb, &bars->full[st]);
                                ++issued;
                                if (++st == NST) { st = 0; ph ^= 1; }
                                if (!b_done && ++sidx == NST && !load_b()) { fail(); goto producer_done; }
                            }
                }
                if (!b_done && !load_b()) { fail(); goto producer_done; }
            }
        producer_done:
            // no copy may be in flight when the CTA exits: wait for the last
            // phase issued on every stage and on the resident B blocks
            // (bounded; earlier phases completed before the buffer was reused)
            for (int q = 0; q < NST && q < issued; ++q) {
                const int last = issued - 1 - q;                 // issue index of a recent copy
                mbar_wait(&bars->full[last % NST], (uint32_t)((last / NST) & 1));
            }
            if (b_issued) mbar_wait(&bars->bfull, (uint32_t)((b_issued - 1) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int st = 0, acc = 0;
            uint32_t ph = 0, aph = 0, bph = 0;
            bool ok = true;
            for (long long it = blockIdx.x; it < a.nitems && !*abort && ok; it += gridDim.x) {
                const Units<MODE> u = item_units<MODE>(a, njt, it);
                if (MODE == 2) {
                    if (!mbar_wait_ab(&bars->bfull, bph, abort)) { fail(); break; }
                    bph ^= 1;
                }
                for (int un = 0; un < u.n && ok; ++un) {
                    const int job = u.job(un);
                    const bool off = MODE == 1 && u.mt != u.nt;
                    const TcJob& jd = off ? c_tcoff[job] : job_desc<MODE>(job);
                    const int nterm = off ? off_terms(jd, job) : jd.nterm;
                    if (!mbar_wait_ab(&bars->acc_empty[acc], aph ^ 1, abort)) { fail(); ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * 256);
                    uint32_t accum = 0;
                    for (int pass = 0; pass < 2 && ok; ++pass)
                        for (int tt = 0; tt < nterm && ok; ++tt) {
                            const bool sw = tt >= jd.nterm;
                            const int t = sw ? tt - jd.nterm : tt;
                            // a term of sign -1: the negate-A bit (13) of the instruction descriptor
                            const bool ng = (((jd.neg >> t) & 1u) != 0) != (sw && off_flip(job));
                            const uint32_t neg = ng ? NEG_A : 0u;
                            const uint32_t id = IDESC | neg, id128 = IDESC_N128 | neg;
                            for (int g = 0; g < G; ++g) {
                                if (!mbar_wait_ab(&bars->full[st], ph, abort)) { fail(); ok = false; break; }
                                tc_fence_after();
                                const uint8_t* sa = smem + stage_a<MODE>(st);
                                const uint8_t* sb = MODE == 2 ? smem + jd.fb[t] * SM_B : sa + SM_A;
                                // slice pairs (i, j) of this stage, or the packed K steps 0, 1 (pass 0)
                                // and 2 (pass 1: copied to the stage's front; resident B keeps it at 2)
                                const int npr = pass ? 1 : a.nks ? 2 : 5;
                                if (sw) {
                                    // A role: conj(B_t(y)) from the B-layout block [br | bi] (slices of
                                    // B_BLK); B role: A_t(y') from the A-layout blocks (re, im per slice)
                                    for (int pr = 0; pr < npr; ++pr) {
                                        const int i = pass ? 0 : a.nks ? pr : c_pi[pr], j = pass ? 0 : a.nks ? pr : c_pj[pr];
                                        const uint64_t x_r = sdesc(sa + i * B_BLK * 2, B_LBO, CM_SBO);
                                        const uint64_t x_i = sdesc(sa + i * B_BLK * 2 + (TM / 8) * 128, B_LBO, CM_SBO);
                                        const uint64_t y_r = sdesc(sb + (j * 2 + 0) * A_BLK * 2, A_LBO, CM_SBO);
                                        const uint64_t y_i = sdesc(sb + (j * 2 + 1) * A_BLK * 2, A_LBO, CM_SBO);
                                        mma_bf16(d, x_r, y_r, id128, 1);                 // Re += br ar
                                        mma_bf16(d, x_i, y_i, id128, 1);                 // Re += bi ai
                                        mma_bf16(d + TM, x_r, y_i, id128, 1);            // Im += br ai
                                        mma_bf16(d + TM, x_i, y_r, id128 ^ NEG_A, 1);    // Im -= bi ar
                                    }
                                    mma_commit(&bars->empty[st]);
                                    if (++st == NST) { st = 0; ph ^= 1; }
                                    continue;
                                }
                                for (int pr = 0; pr < npr; ++pr) {
                                    const int i = pass ? 0 : a.nks ? pr : c_pi[pr];
                                    const int j = pass ? (MODE == 2 && a.nks ? 2 : 0) : a.nks ? pr : c_pj[pr];
                                    const uint64_t a_re = sdesc(sa + (i * 2 + 0) * A_BLK * 2, A_LBO, CM_SBO);
                                    const uint64_t a_im = sdesc(sa + (i * 2 + 1) * A_BLK * 2, A_LBO, CM_SBO);
                                    const uint64_t b_ri = sdesc(sb + j * B_BLK * 2, B_LBO, CM_SBO);
                                    const uint64_t b_i = sdesc(sb + j * B_BLK * 2 + (TM / 8) * 128, B_LBO, CM_SBO);
                                    mma_bf16(d, a_re, b_ri, id, accum);              // Re += ar br, Im += ar bi
                                    accum = 1;
                                    mma_bf16(d, a_im, b_i, id128, 1);                // Re += ai bi
                                    mma_bf16(d + TM, a_im, b_ri, id128 ^ NEG_A, 1);  // Im -= ai br
                                }
                                mma_commit(&bars->empty[st]);
                                if (++st == NST) { st = 0; ph ^= 1; }
                            }
                        }
                    if (!ok) break;
                    mma_commit(&bars->acc_full[acc]);
                    if (++acc == 2) { acc = 0; aph ^= 1; }
                }
                // the resident B blocks are free once this item's MMAs complete
                if (MODE == 2 && ok) mma_commit(&bars->bempty);
            }
            // every MMA of this thread has completed before TMEM is released
            mma_commit(&bars->drain);
            mbar_wait(&bars->drain, 0);
        }
    } else if (MODE == 0) {
        const int q = warp & 3;                       // TMEM lane quarter of this warp
        zf* xp = (zf*)(smem + SMP_EPI) + (warp - 2) * 32 * 33;
        const int YB = (a.ny + 7) / 8;
        int acc = 0;
        uint32_t aph = 0;
        for (long long it = blockIdx.x; it < a.nitems && !*abort; it += gridDim.x) {
            const Units<MODE> u = item_units<MODE>(a, njt, it);
            const int k = u.k, job = u.job(0), mt = u.mt, nt = u.nt;
            if (!mbar_wait_ab(&bars->acc_full[acc], aph, abort)) { fail(); break; }
            tc_fence_after();
            const uint32_t tbase = tmem + (uint32_t)(acc * 256) + ((uint32_t)(q * 32) << 16);
            for (int c = 0; c < 4; ++c) {
                uint32_t re[32], im[32];
                tmem_ld32(tbase + c * 32, re);
                tmem_ld32(tbase + 128 + c * 32, im);
                tmem_ld_wait();
                #pragma unroll
                for (int j = 0; j < 32; ++j) xp[lane * 33 + j] = mk(__uint_as_float(re[j]), __uint_as_float(im[j]));
                __syncwarp();
                const int e = 2 * lane, r8 = e >> 3, c8 = e & 7;
                #pragma unroll
                for (int rg = 0; rg < 4; ++rg) {
                    const int yb = (mt * TM + q * 32) / 8 + rg;
                    #pragma unroll
                    for (int cg = 0; cg < 4; ++cg) {
                        const int ypb = (nt * TM + c * 32) / 8 + cg;
                        if (yb < YB && ypb < YB) {
                            const zf a0 = xp[(8 * rg + r8) * 33 + 8 * cg + c8];
                            const zf a1 = xp[(8 * rg + r8) * 33 + 8 * cg + c8 + 1];
                            float4* dst = (float4*)(a.raw + ((((long long)job * YB + yb) * YB + ypb) * a.Kc + k) * 64 + e);
                            __stcs(dst, make_float4(a0.x, a0.y, a1.x, a1.y));
                        }
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars->acc_empty[acc]);
            if (++acc == 2) { acc = 0; aph ^= 1; }
        }
    } else {
        const int q = warp & 3;                       // TMEM lane quarter of this warp
        const int et = threadIdx.x - 64;              // 0..127 over the epilogue warps
        float2* blk = (float2*)(smem + SMP_EPI);      // EPI_BLOCKS swizzled 32 x 32 blocks
        const float* s_dup = (const float*)(smem + SMP_DUP);
        volatile int* eok = &bars->eok;
        const int cov = a.cov, ny = a.ny;
        const int y = 32 * q + lane;                  // this thread's row of the tile
        int acc = 0;
        uint32_t aph = 0;
        bool go = true;
        for (long long it = blockIdx.x; it < a.nitems && go; it += gridDim.x) {
            const Units<MODE> u = item_units<MODE>(a, njt, it);
            const int k = u.k;
            for (int un = 0; un < u.n; ++un) {
            const int job = u.job(un);
            // one thread waits, so the four warps take the same decision; the
            // barrier also orders this item's block writes after every warp's
            // reads of the previous item
            if (et == 0) *eok = mbar_wait_ab(&bars->acc_full[acc], aph, abort) ? 1 : 0;
            epi_sync();
            const bool ok = *eok != 0;
            epi_sync();
            if (!ok) { if (et == 0) fail(); go = false; break; }
            tc_fence_after();
            const uint32_t tbase = tmem + (uint32_t)(acc * 256) + ((uint32_t)(q * 32) << 16);
            zf* outp = a.out + ((long long)job * a.Kc + k) * a.npp;
            // the item's tiles: rows y0 + [0, 128), columns y1 + [0, 128)
            const int y0 = u.mt * TM, y1 = u.nt * TM, yg = y0 + y;
            // pair_index(yg, y') = rb + y' for this thread's row (32-bit: pairs < 2^31)
            const int rb = (int)(pair_index(yg, yg, ny) - yg);
            if (u.mt != u.nt) {
                // off-diagonal tile pair: the accumulator is the plane up to its
                // scale (A -2, phi 1/2, else 1); each warp stages its rows in
                // its own block for row-contiguous stores
                const float al = job == PL_A ? -2.f : job == PL_PHI ? 0.5f : 1.f;
                float2* bb = blk + q * 1024;
                for (int b = 0; b < 4; ++b) {
                    uint32_t re[32], im[32];
                    tmem_ld32(tbase + b * 32, re);
                    tmem_ld32(tbase + TM + b * 32, im);
                    tmem_ld_wait();
                    __syncwarp();
                    #pragma unroll
                    for (int j = 0; j < 32; ++j)
                        bb[swz(lane, j)] = make_float2(al * __uint_as_float(re[j]), al * __uint_as_float(im[j]));
                    __syncwarp();
                    const int yp = y1 + 32 * b + lane;
                    #pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        const float2 o = bb[swz(r, lane)];
                        const int base = __shfl_sync(0xffffffffu, rb, r);
                        if (y0 + 32 * q + r < cov && yp < cov) __stcs((float2*)(outp + base + yp), o);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars->acc_empty[acc]);
                if (++acc == 2) { acc = 0; aph ^= 1; }
                continue;
            }
            const float dy = s_dup[yg];
            // lay out the blocks (q, c), c <= q
            for (int c = 0; c <= q; ++c) {
                uint32_t re[32], im[32];
                tmem_ld32(tbase + c * 32, re);
                tmem_ld32(tbase + TM + c * 32, im);
                tmem_ld_wait();
                float2* bb = blk + tri_slot(q, c) * 1024;
                #pragma unroll
                for (int j = 0; j < 32; ++j) bb[swz(lane, j)] = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
                if (c < q) bar_arrive64(pair_bar(q, c));
                else __syncwarp();
            }
            // output blocks (q, b), b >= q
            for (int b = q; b < 4; ++b) {
                if (b > q) bar_sync64(pair_bar(b, q));
                float2* bb = blk + tri_slot(b, q) * 1024;     // X(y', y): row y' - 32 b, column y - 32 q
                uint32_t re[32], im[32];
                tmem_ld32(tbase + b * 32, re);
                tmem_ld32(tbase + TM + b * 32, im);
                tmem_ld_wait();
                // out = al X + be conj(X(y', y)): A (-2, 0), S4 / Phi_y / S6 (1, -1),
                // phi (1/2, 1/2), xi (2 U'(y'), 2 U'(y))
                float2 o[32];
                if (job == PL_XI) {
                    #pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float2 pv = bb[swz(j, lane)];
                        const float al = s_dup[y0 + 32 * b + j];
                        o[j] = make_float2(al * __uint_as_float(re[j]) + dy * pv.x,
                                           al * __uint_as_float(im[j]) - dy * pv.y);
                    }
                } else {
                    const float al = job == PL_A ? -2.f : job == PL_PHI ? 0.5f : 1.f;
                    const float be = job == PL_A ? 0.f : job == PL_PHI ? 0.5f : -1.f;
                    #pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float2 pv = bb[swz(j, lane)];
                        o[j] = make_float2(al * __uint_as_float(re[j]) + be * pv.x,
                                           al * __uint_as_float(im[j]) - be * pv.y);
                    }
                }
                __syncwarp();                                  // the block is consumed: it stages the outputs
                #pragma unroll
                for (int j = 0; j < 32; ++j) bb[swz(lane, j)] = o[j];
                __syncwarp();
                // row r of the block: pairs (y0 + 32 q + r, y0 + 32 b + lane),
                // consecutive pair indices rb(y0 + 32 q + r) + y0 + 32 b + lane
                const int yp = y0 + 32 * b + lane;
                #pragma unroll
                for (int r = 0; r < 32; ++r) o[r] = bb[swz(r, lane)];
                if (b > q && y0 + 32 * b + 32 <= cov) {       // whole block above the diagonal
                    #pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        const int base = __shfl_sync(0xffffffffu, rb, r);
                        __stcs((float2*)(outp + base + yp), o[r]);
                    }
                } else {
                    #pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        const int base = __shfl_sync(0xffffffffu, rb, r);
                        const int yr = y0 + 32 * q + r;
                        if (yr < cov && yp >= yr && yp < cov) __stcs((float2*)(outp + base + yp), o[r]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars->acc_empty[acc]);
            if (++acc == 2) { acc = 0; aph ^= 1; }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS_P) : "memory");
    }
}

// ------------------------------------------- edge rows / columns (FP32)
// Entries with y >= cov or y' >= cov (the last row / column of a 128 m + 1
// grid), FP32 products and sums on the CUDA cores, same coefficients.  A term
// of a row-edge entry has the factor conj(A[s][y]) with y on the edge row, a
// term of a column-edge entry the factor B[s][y']; where that factor is zero
// for every snapshot the term is skipped (exact: it adds zeros).  With
// no-slip walls (u = v = w = 0) only the p-v row survives.
__global__ void k_corr_edge(const zf* __restrict__ Xop, int ns, int ny, int Nk, int k0, int Kc, int cov,
                            unsigned jobs, zf* __restrict__ raw)
{
    __shared__ int nz_edge[NFIELD][4];       // field f has a nonzero value on edge row cov + i (i < 4)
    const int kl = blockIdx.x, k = k0 + kl;
    const int ne = ny - cov;
    for (int i = threadIdx.x; i < NFIELD * 4; i += blockDim.x) nz_edge[i / 4][i % 4] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < NFIELD * ns * ne; i += blockDim.x) {
        const int f = i / (ns * ne), r = i - f * ns * ne, s = r / ne, d = r - s * ne;
        const zf v = Xop[(((long long)f * Nk + k) * ns + s) * ny + cov + d];
        if ((v.x != 0.f || v.y != 0.f) && d < 4) atomicOr(&nz_edge[f][d], 1);
    }
    __syncthreads();
    const int n_row = ne * ny, n_col = cov * ne;
    const int YB = (ny + 7) / 8;
    for (int e2 = threadIdx.x; e2 < NJOB * (n_row + n_col); e2 += blockDim.x) {
        const int job = e2 / (n_row + n_col), e = e2 - job * (n_row + n_col);
        int y, yp;
        const bool row_edge = e < n_row;
        if (row_edge) { y = cov + e / ny; yp = e % ny; }
        else { int r = e - n_row; y = r / ne; yp = cov + r % ne; }
        if ((job == NJSQ && yp < y) || !((jobs >> job) & 1u)) continue;
        const TcJob jd = c_tcjobs[job];
        float sr = 0.f, si = 0.f;
        for (int t = 0; t < jd.nterm; ++t) {
            const int d = row_edge ? y - cov : yp - cov;
            if (d < 4 && !nz_edge[row_edge ? jd.fa[t] : jd.fb[t]][d]) continue;   // zero factor
            const zf* A = Xop + ((long long)jd.fa[t] * Nk + k) * ns * ny;
            const zf* B = Xop + ((long long)jd.fb[t] * Nk + k) * ns * ny;
            for (int s = 0; s < ns; ++s) {
                const zf a = A[(long long)s * ny + y], b = B[(long long)s * ny + yp];
                const float ar = a.x, ai = a.y;
                sr = fmaf(ar, b.x, fmaf(ai, b.y, sr));
                si = fmaf(ar, b.y, fmaf(-ai, b.x, si));
            }
        }
        raw[raw_index(job, kl, y, yp, Kc, YB)] = mk(sr, si);
    }
}

// Plane mode: the pairs (y, y') with y' >= cov (the wall row of a 128 m + 1
// grid), in FP32 on the CUDA cores, with the plane definitions of the
// tensor-core epilogue.  X = X(y, y') has the factor B[s][y'] on the edge row,
// X^H needs X(y', y) with the factor conj(A[s][y']) there; terms whose edge
// factor is zero for every snapshot are skipped (exact).  With no-slip walls
// only the pressure term of the phi plane survives.
__global__ void __launch_bounds__(256)
k_corr_edge_planes(const zf* __restrict__ Xop, int ns, int ny, int Nk, int k0, int Kc, int cov,
                   unsigned planes, long long npp, const double* __restrict__ prof, zf* __restrict__ out)
{
    // one warp per wavenumber, eight per CTA
    __shared__ unsigned s_nz[8][NFIELD];     // bit d: the field is nonzero on edge row cov + d (d < 4)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kl = blockIdx.x * 8 + warp;
    if (kl >= Kc) return;
    const int k = k0 + kl;
    const int ne = ny - cov;
    for (int f = 0; f < NFIELD; ++f) {
        unsigned bits = 0;
        for (int i = lane; i < ns * ne; i += 32) {
            const int s2 = i / ne, d = i - s2 * ne;
            const zf v = Xop[(((long long)f * Nk + k) * ns + s2) * ny + cov + d];
            if ((v.x != 0.f || v.y != 0.f) && d < 4) bits |= 1u << d;
        }
        for (int o = 16; o; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        if (lane == 0) s_nz[warp][f] = bits;
    }
    __syncwarp();
    auto nz_edge = [&](int f, int d) -> bool { return (s_nz[warp][f] >> d) & 1u; };
    // edge pairs (y, y'), y <= y', y' in [cov, ny): ne * cov + ne (ne + 1) / 2 of them
    const int n_edge = ne * cov + ne * (ne + 1) / 2;
    for (int e2 = lane; e2 < NPLANE * n_edge; e2 += 32) {
        const int pl = e2 / n_edge;
        int e = e2 - pl * n_edge;
        if (!((planes >> pl) & 1u)) continue;
        int y, yp;
        if (e < ne * cov) { y = e / ne; yp = cov + e % ne; }
        else {
            e -= ne * cov;
            y = cov;
            while (e >= ny - y) { e -= ny - y; ++y; }
            yp = y + e;
        }
        const TcJob jd = c_tcplanes[pl];
        // s1 = X(y, y'), s2 = X(y', y)
        float s1r = 0.f, s1i = 0.f, s2r = 0.f, s2i = 0.f;
        for (int t = 0; t < jd.nterm; ++t) {
            const float c = (((jd.neg >> t) & 1u) ? -1.f : 1.f) * (jd.fa[t] == F_P ? 4.f : 1.f);
            const zf* A = Xop + ((long long)jd.fa[t] * Nk + k) * ns * ny;
            const zf* B = Xop + ((long long)jd.fb[t] * Nk + k) * ns * ny;
            // a factor on an edge row that is zero for every snapshot zeroes the term
            const int d = yp - cov, dy = y - cov;
            const bool ye = dy >= 0 && dy < 4;
            const bool z1 = (d < 4 && !nz_edge(jd.fb[t], d)) || (ye && !nz_edge(jd.fa[t], dy));
            const bool z2 = (d < 4 && !nz_edge(jd.fa[t], d)) || (ye && !nz_edge(jd.fb[t], dy));
            float ar, ai, br, bi;
            if (!z1) {
                float tr = 0.f, ti = 0.f;
                for (int s = 0; s < ns; ++s) {
                    const zf av = A[(long long)s * ny + y], bv = B[(long long)s * ny + yp];
                    ar = av.x; ai = av.y; br = bv.x; bi = bv.y;
                    tr = fmaf(ar, br, fmaf(ai, bi, tr));
                    ti = fmaf(ar, bi, fmaf(-ai, br, ti));
                }
                s1r = fmaf(c, tr, s1r);
                s1i = fmaf(c, ti, s1i);
            }
            if (!z2) {
                float tr = 0.f, ti = 0.f;
                for (int s = 0; s < ns; ++s) {
                    const zf av = A[(long long)s * ny + yp], bv = B[(long long)s * ny + y];
                    ar = av.x; ai = av.y; br = bv.x; bi = bv.y;
                    tr = fmaf(ar, br, fmaf(ai, bi, tr));
                    ti = fmaf(ar, bi, fmaf(-ai, br, ti));
                }
                s2r = fmaf(c, tr, s2r);
                s2i = fmaf(c, ti, s2i);
            }
        }
        zf v;
        if (pl == PL_A) v = mk(-2.f * s1r, -2.f * s1i);
        else if (pl == PL_PHI) v = mk(0.5f * (s1r + s2r), 0.5f * (s1i - s2i));
        else if (pl == PL_XI) {
            const float dy = 2.f * (float)prof[PR_DU * ny + y], dyp = 2.f * (float)prof[PR_DU * ny + yp];
            v = mk(dyp * s1r + dy * s2r, dyp * s1i - dy * s2i);
        } else v = mk(s1r - s2r, s1i + s2i);
        const long long p = pair_index(y, yp, ny);
        out[((long long)pl * Kc + kl) * npp + p] = v;
    }
}

// ------------------------------------------------------------------- host
static void tile_geometry(int ny, int& MT, int& cov)
{
    if (ny > 1 && (ny - 1) % TM == 0) { MT = (ny - 1) / TM; cov = ny - 1; }
    else { MT = (ny + TM - 1) / TM; cov = ny; }
}

// operand slices for Kc wavenumbers (one chunk)
gke_status split_alloc(SplitWork& w, int ny, int ns, int Kc)
{
    const int Nk = Kc;

    int MT, cov;
    tile_geometry(ny, MT, cov);
    const int G = (ns + KS - 1) / KS;
    w.a_bytes = (size_t)Nk * NFIELD * G * MT * A_STAGE * sizeof(bf16);
    w.b_bytes = (size_t)Nk * NFB * G * MT * B_STAGE * sizeof(bf16);
    if (cudaMalloc(&w.ops, w.a_bytes + w.b_bytes) != cudaSuccess) { w.ops = nullptr; return GKE_ERR_OOM; }
    if (cudaMalloc((void**)&w.err, sizeof(int)) != cudaSuccess) { w.err = nullptr; return GKE_ERR_OOM; }
    if (cudaMemset(w.err, 0, sizeof(int)) != cudaSuccess) return GKE_ERR_CUDA;
    w.ops_bytes = w.a_bytes + w.b_bytes;
    return GKE_OK;
}

cudaError_t split_setup(cudaStream_t st)
{
    TcJob h[NJSQ + 1] = {
        /* E  */ {1, {F_U}, {F_V}, 0u},
        /* F  */ {1, {F_P}, {F_V}, 0u},
        /* GX */ {4, {F_Q, F_UU, F_UV, F_UW}, {F_U, F_U, F_V, F_W}, 0u},
        /* QV */ {1, {F_Q}, {F_V}, 0u},
        /* X2 */ {3, {F_UV, F_VV, F_VW}, {F_U, F_V, F_W}, 0u},
        /* GZ */ {4, {F_Q, F_UW, F_VW, F_WW}, {F_W, F_U, F_V, F_W}, 0u},
        /* D  */ {3, {F_U, F_V, F_W}, {F_U, F_V, F_W}, 0u},
    };
    // planes (see the epilogue of k_corr_tc_pipe); B fields are u, v, w
    // (indices 0, 1, 2 of the B operands); the pressure operand of the phi
    // plane is split from 4 p (k_split_prep_A with pscale = 4)
    TcJob hp[NPLANE] = {
        /* A   : D  */ {3, {F_U, F_V, F_W}, {F_U, F_V, F_W}, 0u},
        /* S4  : Gx */ {4, {F_Q, F_UU, F_UV, F_UW}, {F_U, F_U, F_V, F_W}, 0u},
        /* PHIY: Gy */ {4, {F_Q, F_UV, F_VV, F_VW}, {F_V, F_U, F_V, F_W}, 0u},
        /* S6  : Gz */ {4, {F_Q, F_UW, F_VW, F_WW}, {F_W, F_U, F_V, F_W}, 0u},
        /* PHI : H  */ {5, {F_Q, F_UV, F_VV, F_VW, F_P}, {F_V, F_U, F_V, F_W, F_V}, 0x1Eu},
        /* XI  : E  */ {1, {F_U}, {F_V}, 0u},
    };
    // off-diagonal tile pairs: xi = sum conj(u(y)) [2 U'(y') v(y')] + partner,
    // B slot 3 = 2 U'(y) v
    TcJob ho[NPLANE];
    for (int i = 0; i < NPLANE; ++i) ho[i] = hp[i];
    ho[PL_XI].fb[0] = 3;
    static_assert(F_U == 0 && F_V == 1 && F_W == 2, "B operands are u, v, w in field order");
    cudaError_t e = cudaMemcpyToSymbolAsync(c_tcjobs, h, sizeof(h), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_tcplanes, hp, sizeof(hp), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_tcoff, ho, sizeof(ho), 0, cudaMemcpyHostToDevice, st);
    const void* ks[] = {(const void*)k_corr_tc_pipe<0>, (const void*)k_corr_tc_pipe<1>, (const void*)k_corr_tc_pipe<2>};
    for (const void* k : ks)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMP_TOTAL);
    return e;
}

bool split_planes_ok(int ny)
{
    int MT, cov;
    tile_geometry(ny, MT, cov);
    return MT <= DUP_ROWS / TM;
}

static int sm_count()
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return std::max(nsm, 1);
}

// BF16 slices of the operands of wavenumbers [k0, k0 + Kc)
// nfb: B slots written (3: u, v, w; 4: also 2 U'(y) v, which prof gives)
static void split_prep(SplitWork& w, const zf* Xop, int ns, int ny, int Nk, int k0, int Kc, float pscale, int nfb,
                       const double* prof, cudaStream_t st, bf16*& Aop, bf16*& Bop, int& G, int& MT, int& cov,
                       int& nks)
{
    tile_geometry(ny, MT, cov);
    G = (ns + KS - 1) / KS;
    nks = ns <= PK_MAX_NS ? PK_STEPS : 0;
    Aop = (bf16*)w.ops;
    Bop = (bf16*)((char*)w.ops + (size_t)Kc * NFIELD * G * MT * A_STAGE * sizeof(bf16));
    k_split_prep_A<<<(unsigned)((long long)Kc * NFIELD * G * MT), 2 * TM, 0, st>>>(Xop, ns, ny, Nk, k0, G, MT, cov,
                                                                                    pscale, nks, Aop);
    k_split_prep_B<<<(unsigned)((long long)Kc * nfb * G * MT), 2 * TM, 0, st>>>(Xop, ns, ny, Nk, k0, G, MT, cov, nfb,
                                                                                 prof, nks, Bop);
}

// wavenumbers [k0, k0 + Kc) of Nk; raw holds the chunk (raw_index with Kc)
gke_status split_correlate(SplitWork& w, const zf* Xop, int ns, int ny, int Nk, int k0, int Kc, zf* raw,
                           unsigned jobs, cudaStream_t st, std::string& err, int* launches)
{
    *launches = 0;
    TcSel sel{};
    for (int j = 0; j < NJSQ; ++j)
        if ((jobs >> j) & 1u) sel.sq |= (unsigned)j << (3 * sel.nsq++);
    sel.d = (jobs >> J_D) & 1u;
    if (sel.nsq == 0 && !sel.d) return GKE_OK;
    TcArgs a{};
    bf16 *Aop, *Bop;
    split_prep(w, Xop, ns, ny, Nk, k0, Kc, 1.f, 3, nullptr, st, Aop, Bop, a.G, a.MT, a.cov, a.nks);
    a.Aop = Aop; a.Bop = Bop; a.Kc = Kc; a.ny = ny;
    a.sel = sel; a.raw = raw; a.err = w.err;
    a.nitems = (long long)Kc * sel_tiles(sel, a.MT);
    const unsigned grid = (unsigned)std::min<long long>(a.nitems, sm_count());
    k_corr_tc_pipe<0><<<grid, TCP_THREADS, SMP_TOTAL, st>>>(a);
    *launches = 3;
    if (a.cov < ny) {
        k_corr_edge<<<Kc, 256, 0, st>>>(Xop, ns, ny, Nk, k0, Kc, a.cov, jobs, raw);
        *launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { err = std::string("split correlator launch: ") + cudaGetErrorString(e); return GKE_ERR_CUDA; }
    return GKE_OK;
}

// plane mode (split_planes_ok(ny)): the term spectra of the selected planes
// for wavenumbers [k0, k0 + Kc) into out[plane][Kc][npp]
gke_status split_correlate_planes(SplitWork& w, const zf* Xop, int ns, int ny, int Nk, int k0, int Kc,
                                  unsigned planes, long long npp, const double* prof, zf* out, cudaStream_t st,
                                  std::string& err, int* launches)
{
    *launches = 0;
    planes &= (1u << NPLANE) - 1u;
    if (!planes) return GKE_OK;
    if (!split_planes_ok(ny)) { err = "split correlator: plane mode covers at most 4 tiles of 128 rows"; return GKE_ERR_UNSUPPORTED; }
    TcArgs a{};
    bf16 *Aop, *Bop;
    int MT0, cov0;
    tile_geometry(ny, MT0, cov0);
    // off-diagonal tile pairs take the xi plane from the 2 U'(y) v slot
    split_prep(w, Xop, ns, ny, Nk, k0, Kc, 4.f, MT0 > 1 ? 4 : 3, prof, st, Aop, Bop, a.G, a.MT, a.cov, a.nks);
    a.Aop = Aop; a.Bop = Bop; a.Kc = Kc; a.ny = ny;
    a.planes = planes; a.npl = __builtin_popcount(planes); a.npp = npp; a.out = out; a.prof = prof;
    a.ntp = a.MT * (a.MT + 1) / 2;
    a.err = w.err;
    // one tile and one snapshot group: one item per wavenumber with the B
    // blocks resident (each B block is read once per wavenumber); else one
    // item per (wavenumber, tile pair, plane)
    const bool resident = a.G == 1 && a.MT == 1;
    a.nitems = resident ? (long long)Kc : (long long)Kc * a.ntp * a.npl;
    const unsigned grid = (unsigned)std::min<long long>(a.nitems, sm_count());
    if (resident)
        k_corr_tc_pipe<2><<<grid, TCP_THREADS, SMP_TOTAL, st>>>(a);
    else
        k_corr_tc_pipe<1><<<grid, TCP_THREADS, SMP_TOTAL, st>>>(a);
    *launches = 3;
    if (a.cov < ny) {
        k_corr_edge_planes<<<(Kc + 7) / 8, 256, 0, st>>>(Xop, ns, ny, Nk, k0, Kc, a.cov, planes, npp, prof, out);
        *launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { err = std::string("split correlator launch: ") + cudaGetErrorString(e); return GKE_ERR_CUDA; }
    return GKE_OK;
}

gke_status split_check(SplitWork& w, cudaStream_t st, std::string& err)
{
    if (!w.err) return GKE_OK;
    int h = 0;
    if (cudaMemcpyAsync(&h, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        err = "split correlator: cannot read the error flag";
        return GKE_ERR_CUDA;
    }
    if (h) { err = "split correlator: a tensor-core pipeline wait timed out"; return GKE_ERR_CUDA; }
    return GKE_OK;
}

void split_free(SplitWork& w)
{
    if (w.ops) cudaFree(w.ops);
    if (w.err) cudaFree(w.err);
    w.ops = nullptr;
    w.err = nullptr;
}

}  // namespace gke
