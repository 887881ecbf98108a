// spect_internal.cuh -- plan state, device helpers and kernel launchers shared
// by the translation units of the sm_103a SPECT projector library.
//
// Operator (Section II-A of arXiv 2301.09710, Algorithms 1 and 2):
//   A : rotate x and mu by theta_l (bilinear, zero padding), weight by the
//       Eq. (1) accumulated attenuation, blur every depth plane j with
//       p(:,:,j,l) (convolution, replicate padding), sum over depth.
//   A': the exact transpose of every step, in gather (owner-computes) form.
//
// Work layout.  Views are processed in chunks of `chunk` views through one
// work slab of chunk * nx*ny*nz floats laid out [v][k][j][i] (i fastest):
// row (k, j) of view v is contiguous, plane (i, j) of slice k is contiguous.
//   forward : K1 rotate+attenuate  x -> slab (w)      then K2 blur+depth-sum slab -> v
//   back    : K2T blur-adjoint+attenuate v -> slab (t) then K1T adjoint-rotate+view-sum slab -> x
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/spect.h"

namespace spect {

// Per-view rotation constants.  cos/sin are split as hi + lo with hi a
// multiple of 2^-h (h chosen per plan) so that hi * (i - c) + hi' * (j - c)
// is exact in FP32; the fractional sample offset is then formed without
// ever rounding the (large) sample coordinate itself.  See rot_sample().
struct ViewRot {
    float ct_hi, ct_lo, st_hi, st_lo;
};

struct Geometry {
    int nx, ny, nz, nview;
    int px, pz, nvp;  // PSF size and number of PSF views (1 or nview)
    int cint;         // floor((nx-1)/2)
    float cfrac;      // (nx-1)/2 - cint  (0 or 0.5)
    float dy;
    int has_mu;
};

// One adjacency entry of the transposed rotation: source pixel p (i + nx*j
// in the rotated frame) and its bilinear weight on the destination voxel.
struct AdjEntry {
    int p;
    float w;
};

}  // namespace spect

struct spect_plan_s {
    spect::Geometry g;
    int separable;
    int chunk;            // views per slab pass
    int adj_max;          // longest adjacency list
    // device state owned by the plan
    float* mu = nullptr;         // nx*ny*nz
    float* psf = nullptr;        // direct: px*pz*ny*nvp
    float* psf_adj = nullptr;    // direct: nvar * px*pz*ny*nvp edge-class variants for A'
    float* fx = nullptr;         // separable: px*ny*nvp
    float* fz = nullptr;         // separable: pz*ny*nvp
    float* fx_adj = nullptr;     // separable: cls_x * px*ny*nvp
    float* fz_adj = nullptr;     // separable: cls_z * pz*ny*nvp
    spect::ViewRot* rot = nullptr;  // nview
    int* adj_off = nullptr;      // nview*nx*ny + 1
    spect::AdjEntry* adj = nullptr;
    float* slab = nullptr;       // chunk * nx*ny*nz
    size_t slab_cap = 0;         // floats allocated for slab
    size_t part_cap = 0;         // floats allocated for part
    float* e = nullptr;          // nx*ny*nz  (EM back-projection accumulator)
    float* ratio = nullptr;      // nx*nz*nview (EM ratio / ones)
    float* s = nullptr;          // nx*ny*nz  (sensitivity A'1)
    int s_valid = 0;
    int cls_x = 3, cls_z = 3;    // edge classes per axis for A' (1 when the axis has length 1)
    int sep_tk = 0;              // separable kernels: k-rows per block
    // fast path (fused kernels, k-fastest internal layout, cached attenuation)
    cudaStream_t home = nullptr; // creation stream (stream-ordered allocations)
    bool pooled = false;         // memory from cudaMallocAsync (freed with cudaFreeAsync)
    int smem_optin = 0;          // shared memory a block may opt in to (bytes)
    int fast = 0;                // 1 when the fused kernels serve this plan
    int bucket = 0;              // padded tap count of the fused kernels
    int fused_J = 8;             // depth planes per fused forward block
    int fused_nT = 1;            // column tiles per plane in the fused kernels
    int adj_J = 8;               // depth planes per fused adjoint block
    int adj_chunk = 0;           // views per adjoint pass (t slab sized to stay in L2)
    int adj_chunk_req = 0;       // views per adjoint pass asked for (SPECT_ADJ_CHUNK), 0: all
    float* mubar = nullptr;      // nview * ny*nx*nz, [l][j][i][k]
    float* xt = nullptr;         // nx*ny*nz, [j][i][k] image
    float* et = nullptr;         // nx*ny*nz, [j][i][k] back-projection accumulator
    float* st = nullptr;         // nx*ny*nz, [j][i][k] sensitivity
    float* ut = nullptr;         // nx*ny*nz, [j][i][k] regulariser target of the regularised EM
    float* part = nullptr;       // G * nx*nz*nview forward partial sums
    spect::AdjEntry* adjf = nullptr;  // nview*nx*ny*adj_max fixed-length lists
    // patch-staged adjoint gather (gather.cu); gather == 0: the list gather k_adj_rot_t
    int gather = 0;
    int4* gboxes = nullptr;      // [patch][l] source box (i0, j0, width, height)
    spect::AdjEntry* gent = nullptr;  // [patch][l][64][adj_max] box-local entries
    int gbw = 0, gbh = 0, gnpx = 0, gnpy = 0;
    // patch-staged forward rotation (rotpatch.cu): available when rotpatch != 0,
    // used instead of k_rot_fwd when rotpatch_on != 0 (chosen by the autotuner)
    int rotpatch = 0;
    int rotpatch_on = 0;
    // SPECT_PLAN_RECOMPUTE_ATTENUATION: mubar holds the factors of one view
    // chunk (views l0 .. l0+chunk-1 at chunk-relative positions), recomputed
    // from mut (mu in the [j][i][k] layout) before each chunk's kernels
    int recompute = 0;
    float* mut = nullptr;
    size_t mubar_cap = 0;        // floats allocated for mubar
    // three-pass rotation (rot3.cu): the eight-tap table of the forward
    // rotation, [l][j] blocks of rot3_ts8(nx) floats (the adjoint's lists
    // are in adjf)
    int rot3 = 0;
    float* r3_tab = nullptr;
    int4* rboxes = nullptr;      // [patch][l] source box of x_t (i0, j0, width, height)
    int rbw = 0, rbh = 0;
    CUtensorMap rmap_x, rmap_mu; // x_t (k, i, j) and the attenuation cache (k, i, plane)
    int ps = 0;                  // plane stride of the attenuation cache and slab: nx*nz rounded up to 4
    int ts = 0;                  // rotation table block per (view, row): 5*nx rounded up to 4
    float* rtab = nullptr;       // nview*ny*ts rotation tables of the fused forward
    int* err = nullptr;          // device error word (SPECT_ETIMEOUT when a bounded wait ran out)
    size_t bytes = 0;
    // launch accounting and optional per-launch event timing
    long long launches[SPECT_K_COUNT] = {0, 0, 0, 0, 0};
    double prof_ms[SPECT_K_COUNT] = {0, 0, 0, 0, 0};
    int prof = 0;
    struct Pending { int kind; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> evpool;
};

namespace spect {

// --------------------------------------------------------------------- device helpers
// Bilinear sample of rotated-frame pixel (i, j): integer corner (i0, j0) and
// fractional offsets (fx, fy) in [0,1], computed identically by A, by the
// adjacency builder of A', and by the attenuation passes, so the weights of
// A and A' are bitwise the same.  Intrinsics forbid FMA contraction.
struct Sample {
    int i0, j0;
    float fx, fy;
};

__device__ __forceinline__ Sample rot_sample(int i, int j, const ViewRot r, int cint, float cfrac)
{
    // d = index - c, exact (half-)integers
    const float di = __fsub_rn(__fsub_rn((float)i, (float)cint), cfrac);
    const float dj = __fsub_rn(__fsub_rn((float)j, (float)cint), cfrac);
    // exact parts (hi multiples of 2^-h times small half-integers)
    const float ax = __fadd_rn(__fmul_rn(r.ct_hi, di), __fmul_rn(r.st_hi, dj));
    const float ay = __fsub_rn(__fmul_rn(r.ct_hi, dj), __fmul_rn(r.st_hi, di));
    // small residuals
    const float rx = __fadd_rn(__fmul_rn(r.ct_lo, di), __fmul_rn(r.st_lo, dj));
    const float ry = __fsub_rn(__fmul_rn(r.ct_lo, dj), __fmul_rn(r.st_lo, di));
    const float tx = __fadd_rn(ax, cfrac);  // exact
    const float ty = __fadd_rn(ay, cfrac);
    const float flx = floorf(tx), fly = floorf(ty);
    float fx = __fadd_rn(__fsub_rn(tx, flx), rx);
    float fy = __fadd_rn(__fsub_rn(ty, fly), ry);
    int i0 = (int)flx + cint, j0 = (int)fly + cint;
    if (fx < 0.f) { fx = __fadd_rn(fx, 1.f); i0 -= 1; }
    else if (fx >= 1.f) { fx = __fsub_rn(fx, 1.f); i0 += 1; }
    if (fy < 0.f) { fy = __fadd_rn(fy, 1.f); j0 -= 1; }
    else if (fy >= 1.f) { fy = __fsub_rn(fy, 1.f); j0 += 1; }
    Sample s;
    s.i0 = i0; s.j0 = j0; s.fx = fx; s.fy = fy;
    return s;
}

// Weight of corner (di, dj) in {0,1}^2 of a bilinear sample.
__device__ __forceinline__ float bilinear_w(const Sample& s, int di, int dj)
{
    const float wx = di ? s.fx : __fsub_rn(1.f, s.fx);
    const float wy = dj ? s.fy : __fsub_rn(1.f, s.fy);
    return __fmul_rn(wx, wy);
}

// Bilinear gather from one nx*ny slice with zero padding (Section II-A).
__device__ __forceinline__ float gather_bilinear(const float* __restrict__ sl, const Sample& s, int nx, int ny)
{
    const bool vi0 = (unsigned)s.i0 < (unsigned)nx, vi1 = (unsigned)(s.i0 + 1) < (unsigned)nx;
    const bool vj0 = (unsigned)s.j0 < (unsigned)ny, vj1 = (unsigned)(s.j0 + 1) < (unsigned)ny;
    const float* row0 = sl + (ptrdiff_t)s.j0 * nx + s.i0;
    const float* row1 = row0 + nx;
    float acc = 0.f;
    if (vj0 && vi0) acc = __fmaf_rn(bilinear_w(s, 0, 0), __ldg(row0), acc);
    if (vj0 && vi1) acc = __fmaf_rn(bilinear_w(s, 1, 0), __ldg(row0 + 1), acc);
    if (vj1 && vi0) acc = __fmaf_rn(bilinear_w(s, 0, 1), __ldg(row1), acc);
    if (vj1 && vi1) acc = __fmaf_rn(bilinear_w(s, 1, 1), __ldg(row1 + 1), acc);
    return acc;
}

// Running Eq. (1) attenuation along depth, from the detector side (j = ny-1)
// inwards: S = sum_{s>j} mu~(s) kept with Kahan compensation.
// Eq. (1) as a warp scan along depth.  Lane q of the warp holds mu~ of the
// q-th of 32 consecutive depths counted from the detector side; `carry` is the
// sum of mu~ over every depth nearer the detector (a double-float pair).  The
// inclusive prefix sums over the lanes are formed in five shuffle steps with
// compensated (two-sum) additions, so the sum S of Eq. (1) keeps about twice
// FP32's precision however many depths it spans; the lane's factor is
// exp(-dy (S + mu~/2)) with S the sum over the depths before it.  carry
// advances past the 32 depths.  Every lane of the warp must call it.
struct DFloat {
    float hi, lo;
};

__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    const float hi = s + e;
    return {hi, e - (hi - s)};
}

__device__ __forceinline__ float atten_warp_scan(float m, DFloat& carry, float dy)
{
    const int lane = threadIdx.x & 31;
    DFloat inc = {m, 0.f};
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const DFloat o = {__shfl_up_sync(0xffffffffu, inc.hi, d), __shfl_up_sync(0xffffffffu, inc.lo, d)};
        if (lane >= d) inc = df_add(o, inc);
    }
    DFloat ex = {__shfl_up_sync(0xffffffffu, inc.hi, 1), __shfl_up_sync(0xffffffffu, inc.lo, 1)};
    if (lane == 0) ex = {0.f, 0.f};
    const DFloat sum = df_add(carry, ex);
    const float mb = expf(-dy * (sum.hi + (sum.lo + 0.5f * m)));
    const DFloat tot = {__shfl_sync(0xffffffffu, inc.hi, 31), __shfl_sync(0xffffffffu, inc.lo, 31)};
    carry = df_add(carry, tot);
    return mb;
}

// Eq. (1) walked serially from the detector side with a compensated running
// sum (the low-memory blur adjoints, which visit depths one at a time).
struct AttenScan {
    float S = 0.f, c = 0.f;
    // mubar(j) = exp(-dy (mu~(j)/2 + S)), then S += mu~(j)
    __device__ __forceinline__ float step(float m, float dy)
    {
        const float half = 0.5f * m - c;
        const float mb = expf(-dy * (S + half));
        const float y = m - c;
        const float t = S + y;
        c = (t - S) - y;
        S = t;
        return mb;
    }
};

// EM update of one voxel from its back-projected ratio e (Eqs. (7)-(8)):
// MLEM x e / s when beta == 0; otherwise the non-negative root of
// beta x'^2 + (s - beta u) x' - x e = 0, evaluated in the cancellation-free
// form for the sign of d = s - beta u.  Non-positive denominators give 0.
__device__ __forceinline__ float em_update(float x, float e, float s, float u, float beta)
{
    const float xe = x * e;
    if (beta == 0.f) return s > 0.f ? xe / s : 0.f;
    const float d = fmaf(-beta, u, s);  // explicit: every kernel rounds d the same way
    const float root = sqrtf(fmaf(d, d, 4.f * beta * xe));
    if (d >= 0.f) {
        const float den = d + root;
        return den > 0.f ? (2.f * xe) / den : 0.f;
    }
    return (root - d) / (2.f * beta);
}

// Arguments of the EM epilogue of the adjoint-rotation kernels; x == nullptr
// means plain back-projection.
struct EmArgs {
    float* x = nullptr;        // updated in place
    const float* s = nullptr;  // sensitivity A'1 (same layout as x)
    const float* u = nullptr;  // regulariser target (beta > 0 only)
    float beta = 0.f;
};

// Kahan-compensated accumulator for depth and view sums.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s - c; }
};

// --------------------------------------------------------------------- TMA bulk copies
// 1D bulk copies between global and shared memory (cp.async.bulk) completed
// through an mbarrier.  Every wait is bounded: a wait that runs out returns
// false and the caller records SPECT_ETIMEOUT in the plan's error word.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Start a bulk copy global -> shared whose bytes complete on `bar`.
__device__ __forceinline__ void tma_copy_1d(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst_smem)),
                 "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Arrive on `bar` expecting `bytes` of transaction, then start the copy.
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    tma_copy_1d(dst_smem, src_gmem, bytes, bar);
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` for at most ~2^31 SM clocks (about one second).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < (1ll << 31))
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_store_1d(void* dst_gmem, const void* src_smem, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem), "r"(smem_u32(src_smem)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until at most N committed bulk stores still read their shared-memory source.
template <int N>
__device__ __forceinline__ void tma_store_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// One 4-byte asynchronous copy global -> shared (cp.async, through L1), and the
// wait for all of the calling thread's copies.
__device__ __forceinline__ void cp_async_4(float* dst_smem, const float* src_gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst_smem)), "l"(src_gmem) : "memory");
}

// The same, writing 0.0f instead of reading when !valid (src is not read then).
__device__ __forceinline__ void cp_async_4_or_zero(float* dst_smem, const float* src_gmem, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst_smem)), "l"(src_gmem),
                 "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Row pitch (floats) of the shared-memory plane images: at least n, a multiple of
// 4 with pitch/4 odd, so rows are 16-byte aligned and float4 loads with lanes
// over rows are bank-conflict free.
__host__ __device__ inline int pitch4odd(int n)
{
    int q = (n + 3) / 4;
    if ((q & 1) == 0) ++q;
    return 4 * q;
}

// Tiled 3D tensor load (TMA) of the box at coordinates (c0, c1, c2) of `map`
// into shared memory (128-byte aligned), completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst_smem, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst_smem)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Host: cuTensorMapEncodeTiled through the runtime's driver entry point (NULL when unavailable).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_fn();

// --------------------------------------------------------------------- launchers
// Host: per-view rotation constants for nview angles (NULL: 2 pi l / nview).
void make_view_rot(int nx, int nview, const double* angles, ViewRot* out);
// Host: record `st` and `msg` for spect_last_error() on this thread; returns st.
spect_status set_error(spect_status st, const char* msg);

// All return the cudaError_t of the launch (cudaGetLastError()).
cudaError_t launch_build_adjacency(const spect_plan_s& P, int pass, int* counts, int* maxcount, cudaStream_t st);
cudaError_t launch_rotate_atten(const spect_plan_s& P, const float* x, int l0, int nv, cudaStream_t st);
cudaError_t launch_rotate_adjoint(const spect_plan_s& P, int l0, int nv, float* out, int accumulate, EmArgs em,
                                  cudaStream_t st);
cudaError_t launch_conv_forward(const spect_plan_s& P, float* v, int l0, int nv, const float* em_y,
                                const float* em_rbar, cudaStream_t st);
cudaError_t launch_conv_adjoint(const spect_plan_s& P, const float* v, int l0, int nv, cudaStream_t st);
cudaError_t launch_psf_variants(spect_plan_s& P, float* scratch, cudaStream_t st);
int choose_sep_tile(const Geometry& g, int cls_z, size_t smem_limit);
// fast path (fused.cu)
// PSF bucket (padded tap count) of the fused kernels for this geometry, 0 when
// they do not fit; *tiles receives the column-tile count they need.
int fused_bucket(const Geometry& g, size_t smem_limit, int* tiles);
int fused_groups(const spect_plan_s& P);
// Bucket of the fused full-PSF kernels (untiled planes), 0 when they do not fit.
int fused_dir_bucket(const Geometry& g, size_t smem_limit);
bool fused_dir_fit(const Geometry& g, int bucket, int J, int adj_J, size_t smem_limit);
int fused_tiles_fit(const Geometry& g, int bucket, int J, int adj_J, int tiles, size_t smem_limit);
cudaError_t launch_transpose(const float* in, float* out, int R, int C, cudaStream_t st);
cudaError_t launch_mubar_cache(const spect_plan_s& P, const float* mu_t, cudaStream_t st);
cudaError_t launch_build_adjacency_fixed(const spect_plan_s& P, cudaStream_t st);
cudaError_t launch_rot_tables(const spect_plan_s& P, cudaStream_t st);
cudaError_t launch_fused_forward(const spect_plan_s& P, const float* xt, int l0, int nv, cudaStream_t st);
cudaError_t launch_fused_rotate(const spect_plan_s& P, const float* xt, int l0, int nv, cudaStream_t st);
// three-pass rotation (rot3.cu): table block size, and the plan-time build of
// the table, the adjoint lists (adjf, adj_max >= 8) and the attenuation cache
int rot3_ts8(int nx);
cudaError_t build_rot3(spect_plan_s& P, const double* angles, const float* mu_t, float* scratch, cudaStream_t st);
size_t fused_slab_per_view(const spect_plan_s& P);
cudaError_t launch_fused_adjoint(const spect_plan_s& P, const float* v, int l0, int nv, cudaStream_t st);
cudaError_t launch_fwd_reduce(const spect_plan_s& P, float* v, const float* em_y, const float* em_rbar,
                              cudaStream_t st);
cudaError_t build_gather(spect_plan_s& P, cudaStream_t st);
cudaError_t build_rotpatch(spect_plan_s& P, cudaStream_t st);
cudaError_t launch_rot_patch(const spect_plan_s& P, int l0, int nv, cudaStream_t st);
// the attenuation factors of views l0 .. l0+nv-1 (recomputing plans: into the chunk buffer)
cudaError_t launch_mubar_range(const spect_plan_s& P, int l0, int nv, cudaStream_t st);
// The attenuation array as the kernels index it, mubar + (l ny + j) ps for view l:
// a recomputing plan holds views l0.. at chunk-relative positions, so its base is
// moved back by l0 views (computed on integers; every access lands in the buffer).
inline const float* mubar_for(const spect_plan_s& P, int l0)
{
    if (!P.recompute) return P.mubar;
    return reinterpret_cast<const float*>(reinterpret_cast<uintptr_t>(P.mubar) -
                                          (uintptr_t)l0 * P.g.ny * P.ps * sizeof(float));
}
cudaError_t launch_adj_gather(const spect_plan_s& P, int l0, int nv, float* out, int accumulate, EmArgs em,
                              cudaStream_t st);
cudaError_t launch_adj_rot_t(const spect_plan_s& P, int l0, int nv, float* out, int accumulate, EmArgs em,
                             cudaStream_t st);
bool direct_fits(const Geometry& g, size_t smem_limit);
// grouped launches of a batch of plans (grouped.cu, gather.cu): per stage and
// kernel variant one launch over a work list spanning the plans (at most
// kGroupMax plans per launch); head / iter / tail: layouts in, one EM
// iteration, layouts out
constexpr int kGroupMax = 24;
// Where each plan's blocks sit in a grouped launch: plan m owns blocks
// [first[m], first[m+1]) laid out as its own grid (gx x gy x gz, x fastest),
// so a block finds its plan and coordinates from blockIdx.x alone.
struct GroupGrid {
    int n;
    int first[kGroupMax + 1];
    int gx[kGroupMax], gy[kGroupMax];
};
__device__ __forceinline__ int4 group_item(const GroupGrid& gg)
{
    const int b = (int)blockIdx.x;
    int m = 0;
    while (m + 1 < gg.n && b >= gg.first[m + 1]) ++m;
    const int r = b - gg.first[m], gx = gg.gx[m], gy = gg.gy[m];
    const int q = r / gx;
    return make_int4(m, r - q * gx, q % gy, q / gy);
}
using GroupLaunch = std::function<cudaError_t(cudaStream_t)>;
struct GroupedBatch {
    std::vector<GroupLaunch> head, iter, tail;
};
bool groupable(const spect_plan_s& P);
cudaError_t build_grouped(const std::vector<spect_plan_s*>& plans, float* const* x, const float* const* y,
                          const float* const* rbar, GroupedBatch& B);
cudaError_t build_grouped_gather(const std::vector<spect_plan_s*>& plans, GroupedBatch& B,
                                 std::vector<GroupLaunch>& out);
void free_grouped(GroupedBatch& B);
cudaError_t launch_fill(float* p, size_t n, float value, cudaStream_t st);

}  // namespace spect
