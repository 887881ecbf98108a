// plan.cu -- the C ABI (include/spect.h): plan construction, argument
// validation, and the stream-ordered orchestration of the kernels for
// A (Algorithm 1), A' (Algorithm 2) and the MLEM update (Eqs. (7)-(8), beta=0).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "spect_internal.cuh"

using spect::Geometry;
using spect::ViewRot;

namespace spect {
void make_view_rot(int nx, int nview, const double* angles, ViewRot* out);
}

namespace {

thread_local std::string g_err;

spect_status fail(spect_status st, const std::string& msg)
{
    g_err = msg;
    return st;
}

#define SPECT_CUDA_TRY(expr, what)                                                        \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(SPECT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// cos/sin with exact values at multiples of pi/2 (the rotation of a quarter
// turn is then an exact lattice permutation).
void exact_cos_sin(double th, double* c, double* s)
{
    const double q = th / (M_PI / 2.0);
    const double r = nearbyint(q);
    if (fabs(q - r) < 1e-12) {
        const long m = (((long)r % 4) + 4) % 4;
        *c = (m == 0) ? 1.0 : (m == 2 ? -1.0 : 0.0);
        *s = (m == 1) ? 1.0 : (m == 3 ? -1.0 : 0.0);
    } else {
        *c = cos(th);
        *s = sin(th);
    }
}

// Split t = hi + lo with hi a multiple of 2^-h (see rot_sample()).
void split(double t, int h, float* hi, float* lo)
{
    const double sc = ldexp(1.0, h);
    const double th = nearbyint(t * sc) / sc;
    *hi = (float)th;
    *lo = (float)(t - th);
}

}  // namespace

// Per-view rotation constants (see rot_sample()): cos/sin split into a part
// on a 2^-h grid, h chosen from nx so the products with (i - c) are exact.
void spect::make_view_rot(int nx, int nview, const double* angles, ViewRot* out)
{
    int lg = 0;
    while ((1 << lg) < nx) ++lg;
    const int h = 22 - lg;
    for (int l = 0; l < nview; ++l) {
        const double th = angles ? angles[l] : 2.0 * M_PI * (double)l / (double)nview;
        double c, s;
        exact_cos_sin(th, &c, &s);
        split(c, h, &out[l].ct_hi, &out[l].ct_lo);
        split(s, h, &out[l].st_hi, &out[l].st_lo);
    }
}

namespace {

// Plan memory is stream-ordered (cudaMallocAsync on the creation stream) when
// the device has memory pools, so plans can be created and released while
// other plans' kernels run, without a device-wide synchronisation.
cudaError_t raw_alloc(spect_plan_s* P, void** p, size_t bytes, cudaStream_t st)
{
    return P->pooled ? cudaMallocAsync(p, bytes, st) : cudaMalloc(p, bytes);
}

void raw_free(spect_plan_s* P, void* p, cudaStream_t st)
{
    if (!p) return;
    if (P->pooled) cudaFreeAsync(p, st);
    else cudaFree(p);
}

template <class T>
spect_status dalloc(spect_plan_s* P, T** p, size_t count, const char* what)
{
    *p = nullptr;
    if (count == 0) return SPECT_OK;
    const size_t bytes = count * sizeof(T);
    cudaError_t e = raw_alloc(P, (void**)p, bytes, P->home);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SPECT_ENOMEM : SPECT_ECUDA,
                    std::string("allocating ") + what + ": " + cudaGetErrorString(e));
    }
    // the kernels use 16-byte vector and bulk-copy accesses from these bases
    if (((uintptr_t)*p & 255) != 0) {
        raw_free(P, *p, P->home);
        *p = nullptr;
        return fail(SPECT_ECUDA, std::string("allocation of ") + what + " is not 256-byte aligned");
    }
    P->bytes += bytes;
    return SPECT_OK;
}

void free_plan(spect_plan_s* P, cudaStream_t st)
{
    if (!P) return;
    for (auto& p : P->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : P->evpool) cudaEventDestroy(e);
    void* ptrs[] = {P->mu, P->psf, P->psf_adj, P->fx, P->fz, P->fx_adj, P->fz_adj, P->rot, P->adj_off, P->adj,
                    P->slab, P->e, P->ratio, P->s, P->mubar, P->xt, P->et, P->st, P->part, P->adjf, P->err, P->rtab, P->ut,
                    P->gboxes, P->gent, P->rboxes, P->r3_tab, P->mut};
    for (void* p : ptrs) raw_free(P, p, st);
    delete P;
}

// a plan that failed during creation: its memory is freed on the creation stream
void free_plan(spect_plan_s* P) { free_plan(P, P ? P->home : nullptr); }

size_t slab_budget_bytes(bool fast)
{
    // Work slab size.  The fused path takes every view in one pass when the
    // slab fits 1 GiB; the low-memory path keeps it at 256 MiB.
    // SPECT_SLAB_MB overrides (tuning).
    const char* env = getenv("SPECT_SLAB_MB");
    long mb = env ? atol(env) : (fast ? 1024 : 256);
    if (mb < 1) mb = 1;
    return (size_t)mb << 20;
}

// Budget of a recomputing plan's per-chunk buffers (work slab plus the
// attenuation factors of the chunk's views): 512 MiB, or SPECT_SLAB_MB (tuning).
size_t recompute_budget_bytes()
{
    const char* env = getenv("SPECT_SLAB_MB");
    long mb = env ? atol(env) : 512;
    if (mb < 1) mb = 1;
    return (size_t)mb << 20;
}

// Bytes one view of a chunk takes: its work-slab share, plus its attenuation
// factors when the plan recomputes them per chunk.
size_t view_bytes(const spect_plan_s& P, size_t slab_floats_per_view)
{
    size_t f = slab_floats_per_view;
    if (P.recompute) f += (size_t)P.g.ny * P.ps;
    return f * sizeof(float);
}

// The patch gather reads its own box-local copy of the adjacency entries, so
// once it is set up the fixed-length lists were set-up input only: free them.
void drop_fixed_lists(spect_plan_s* P, cudaStream_t st)
{
    if (!P->gather || !P->adjf) return;
    const size_t nlist = (size_t)P->g.nx * P->g.ny * P->g.nview;
    raw_free(P, P->adjf, st);
    P->adjf = nullptr;
    P->bytes -= nlist * (size_t)std::max(P->adj_max, 1) * sizeof(spect::AdjEntry);
}

cudaEvent_t pool_event(spect_plan_s* P)
{
    if (!P->evpool.empty()) {
        cudaEvent_t e = P->evpool.back();
        P->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Count a launch of kernel class `kind`; when profiling, bracket it with events.
template <class F>
cudaError_t counted(spect_plan_s* P, int kind, cudaStream_t st, F&& launch)
{
    P->launches[kind] += 1;
    if (!P->prof) return launch();
    cudaEvent_t a = pool_event(P), b = pool_event(P);
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaEventRecord(a, st);
    cudaError_t e = launch();
    cudaEventRecord(b, st);
    P->pending.push_back({kind, a, b});
    return e;
}

cudaError_t drain_profile(spect_plan_s* P)
{
    cudaError_t err = cudaSuccess;
    for (auto& p : P->pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) err = e;
        else P->prof_ms[p.kind] += ms;
        P->evpool.push_back(p.a);
        P->evpool.push_back(p.b);
    }
    P->pending.clear();
    return err;
}

spect_status run_forward(spect_plan_s* P, const float* x, float* v, const float* y, const float* rbar,
                         cudaStream_t st)
{
    const int nview = P->g.nview;
    for (int l0 = 0; l0 < nview; l0 += P->chunk) {
        const int nv = std::min(P->chunk, nview - l0);
        SPECT_CUDA_TRY(counted(P, SPECT_K_ROTATE_ATTEN, st, [&] { return spect::launch_rotate_atten(*P, x, l0, nv, st); }),
                       "rotate/attenuate launch");
        SPECT_CUDA_TRY(counted(P, SPECT_K_CONV_FWD, st,
                               [&] { return spect::launch_conv_forward(*P, v, l0, nv, y, rbar, st); }),
                       "PSF blur launch");
    }
    return SPECT_OK;
}

// out = A' v; with em.x set, the last chunk applies the EM update to em.x instead.
spect_status run_back(spect_plan_s* P, const float* v, float* out, spect::EmArgs em, cudaStream_t st)
{
    const int nview = P->g.nview;
    for (int l0 = 0; l0 < nview; l0 += P->chunk) {
        const int nv = std::min(P->chunk, nview - l0);
        const bool last = l0 + nv >= nview;
        SPECT_CUDA_TRY(counted(P, SPECT_K_CONV_ADJ, st, [&] { return spect::launch_conv_adjoint(*P, v, l0, nv, st); }),
                       "PSF blur adjoint launch");
        spect::EmArgs e = em;
        if (!last) e.x = nullptr;
        SPECT_CUDA_TRY(counted(P, SPECT_K_ROTATE_ADJ, st,
                               [&] { return spect::launch_rotate_adjoint(*P, l0, nv, out, l0 > 0, e, st); }),
                       "adjoint rotation launch");
    }
    return SPECT_OK;
}

// ---- fused path: internal volumes in the [j][i][k] layout
spect_status to_internal(spect_plan_s* P, const float* x, float* xt, cudaStream_t st)
{
    const int nxy = P->g.nx * P->g.ny;
    SPECT_CUDA_TRY(counted(P, SPECT_K_OTHER, st, [&] { return spect::launch_transpose(x, xt, P->g.nz, nxy, st); }),
                   "transpose launch");
    return SPECT_OK;
}

spect_status from_internal(spect_plan_s* P, const float* xt, float* x, cudaStream_t st)
{
    const int nxy = P->g.nx * P->g.ny;
    SPECT_CUDA_TRY(counted(P, SPECT_K_OTHER, st, [&] { return spect::launch_transpose(xt, x, nxy, P->g.nz, st); }),
                   "transpose launch");
    return SPECT_OK;
}

// v = A x_t (x_t internal layout); with y set, v receives the EM ratio y / (A x + rbar)
spect_status fast_forward(spect_plan_s* P, const float* xt, float* v, const float* y, const float* rbar,
                          cudaStream_t st)
{
    const int nview = P->g.nview;
    for (int l0 = 0; l0 < nview; l0 += P->chunk) {
        const int nv = std::min(P->chunk, nview - l0);
        if (P->recompute)  // Eq. (1) factors of this chunk's views
            SPECT_CUDA_TRY(counted(P, SPECT_K_ROTATE_ATTEN, st, [&] { return spect::launch_mubar_range(*P, l0, nv, st); }),
                           "attenuation launch");
        SPECT_CUDA_TRY(counted(P, SPECT_K_ROTATE_ATTEN, st,
                               [&] { return spect::launch_fused_rotate(*P, xt, l0, nv, st); }),
                       "rotation launch");
        SPECT_CUDA_TRY(counted(P, SPECT_K_CONV_FWD, st,
                               [&] { return spect::launch_fused_forward(*P, xt, l0, nv, st); }),
                       "fused forward launch");
    }
    SPECT_CUDA_TRY(counted(P, SPECT_K_OTHER, st, [&] { return spect::launch_fwd_reduce(*P, v, y, rbar, st); }),
                   "depth-group reduce launch");
    return SPECT_OK;
}

// out_t = A' v (internal layout); with em.x set the last chunk applies the EM update instead
spect_status fast_back(spect_plan_s* P, const float* v, float* out_t, spect::EmArgs em, cudaStream_t st)
{
    const int nview = P->g.nview;
    for (int l0 = 0; l0 < nview; l0 += P->adj_chunk) {
        const int nv = std::min(P->adj_chunk, nview - l0);
        const bool last = l0 + nv >= nview;
        if (P->recompute)  // Eq. (1) factors of this chunk's views
            SPECT_CUDA_TRY(counted(P, SPECT_K_CONV_ADJ, st, [&] { return spect::launch_mubar_range(*P, l0, nv, st); }),
                           "attenuation launch");
        SPECT_CUDA_TRY(counted(P, SPECT_K_CONV_ADJ, st, [&] { return spect::launch_fused_adjoint(*P, v, l0, nv, st); }),
                       "fused adjoint launch");
        spect::EmArgs e = em;
        if (!last) e.x = nullptr;
        SPECT_CUDA_TRY(counted(P, SPECT_K_ROTATE_ADJ, st,
                               [&] {
                                   return P->gather ? spect::launch_adj_gather(*P, l0, nv, out_t, l0 > 0, e, st)
                                                    : spect::launch_adj_rot_t(*P, l0, nv, out_t, l0 > 0, e, st);
                               }),
                       "adjoint rotation launch");
    }
    return SPECT_OK;
}

spect_status ensure_sensitivity(spect_plan_s* P, cudaStream_t st)
{
    if (P->s_valid) return SPECT_OK;
    const size_t nproj = (size_t)P->g.nx * P->g.nz * P->g.nview;
    SPECT_CUDA_TRY(counted(P, SPECT_K_OTHER, st, [&] { return spect::launch_fill(P->ratio, nproj, 1.f, st); }),
                   "fill launch");
    spect_status r = P->fast ? fast_back(P, P->ratio, P->st, spect::EmArgs(), st)
                             : run_back(P, P->ratio, P->s, spect::EmArgs(), st);
    if (r != SPECT_OK) return r;
    if (P->fast) {
        r = from_internal(P, P->st, P->s, st);
        if (r != SPECT_OK) return r;
    }
    P->s_valid = 1;
    return SPECT_OK;
}

spect_status em_iterate(spect_plan_s* P, float* x, const float* y, const float* rbar, const float* u, float beta,
                        int niter, cudaStream_t st);

spect_status check_call(spect_plan P, const void* a, const void* b, const char* na, const char* nb)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    if (!a) return fail(SPECT_EINVAL, std::string(na) + " is NULL");
    if (!b) return fail(SPECT_EINVAL, std::string(nb) + " is NULL");
    if (!aligned16(a)) return fail(SPECT_EINVAL, std::string(na) + " is not 16-byte aligned");
    if (!aligned16(b)) return fail(SPECT_EINVAL, std::string(nb) + " is not 16-byte aligned");
    return SPECT_OK;
}

}  // namespace

// Record a status and message for spect_last_error() (other translation units).
spect_status spect::set_error(spect_status st, const char* msg) { return fail(st, msg); }

extern "C" {

const char* spect_last_error(void) { return g_err.c_str(); }

const char* spect_version(void) { return "spect-gb300 0.1 (sm_103a)"; }

namespace {

// Upper bound of the device bytes a plan of this geometry allocates (the sum
// of the allocations in spect_plan_create, with the adjacency lists at their
// largest: 8 fixed entries per list, or 4 entries per source pixel in the
// compressed form, whichever is larger).  When the fused kernels serve a
// geometry, their buffers dominate those of the low-memory path it may fall
// back to, so the fused sizes bound both.
size_t plan_bytes_bound(const spect_plan_s& P)
{
    const Geometry& g = P.g;
    const size_t F = sizeof(float);
    const size_t vol = (size_t)g.nx * g.ny * g.nz, nproj = (size_t)g.nx * g.nz * g.nview;
    const size_t nxy = (size_t)g.nx * g.ny, nrows = (size_t)g.nvp * g.ny, nlist = nxy * g.nview;
    size_t b = sizeof(int) + vol * F;
    if (P.separable) b += ((size_t)g.px * 4 + (size_t)g.pz * (1 + P.cls_z)) * nrows * F;
    else b += (size_t)g.px * g.pz * nrows * (1 + (size_t)P.cls_x * P.cls_z) * F;
    b += (size_t)g.nview * sizeof(ViewRot);
    const size_t fixed = nlist * 8 * sizeof(spect::AdjEntry);
    const size_t csr = (nlist + 1) * sizeof(int) + 4 * nlist * sizeof(spect::AdjEntry);
    b += P.fast ? std::max(fixed, csr) : csr;
    const size_t per_view = std::max(vol, P.fast ? spect::fused_slab_per_view(P) : vol);
    const size_t budget = P.recompute ? recompute_budget_bytes() : slab_budget_bytes(P.fast);
    const size_t chunk = std::max<size_t>(1, std::min<size_t>((size_t)g.nview, budget / view_bytes(P, per_view)));
    b += per_view * chunk * F;
    b += (2 * vol + nproj) * F;
    if (P.fast) {
        // attenuation factors of every view, or of one chunk plus mu in the internal layout
        b += P.recompute ? ((size_t)g.ny * P.ps * chunk + vol) * F : (size_t)g.ny * P.ps * g.nview * F;
        b += 4 * vol * F;
        b += nproj * (size_t)spect::fused_groups(P) * F + (size_t)g.nview * g.ny * P.ts * F;
        // patch gather: boxes and box-local entries (at most 8 per list)
        const size_t np = (size_t)((g.nx + 7) / 8) * ((g.ny + 7) / 8) * g.nview;
        b += np * 16 + np * 64 * 8 * sizeof(spect::AdjEntry) + np * 16;  // + rotation boxes
        if (P.rot3)  // the eight-tap table
            b += (size_t)g.nview * g.ny * 16 * (size_t)g.nx * F;
    }
    return b;
}

}  // namespace

spect_status spect_plan_bytes(int nx, int ny, int nz, int nview, int px, int pz, int nview_psf, int separable,
                              unsigned flags, size_t* bytes)
{
    if (!bytes) return fail(SPECT_EINVAL, "bytes is NULL");
    *bytes = 0;
    if (nx != ny || nx < 2 || nx > 1024 || nz < 1 || nz > 4096 || nview < 1 || nview > 4096)
        return fail(SPECT_EINVAL, "geometry out of range (as spect_plan_create)");
    if (px < 1 || pz < 1 || px > 127 || pz > 127 || (px % 2) == 0 || (pz % 2) == 0)
        return fail(SPECT_EINVAL, "PSF sizes px, pz must be odd and in [1, 127]");
    if (nview_psf != 1 && nview_psf != nview) return fail(SPECT_EINVAL, "nview_psf must be 1 or nview");
    int dev = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(SPECT_ECUDA, "device query failed");
    }
    spect_plan_s P;
    Geometry& g = P.g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.nview = nview;
    g.px = px; g.pz = pz; g.nvp = nview_psf;
    P.separable = separable != 0;
    P.ps = (nx * nz + 3) & ~3;
    P.ts = (5 * nx + 3) & ~3;
    P.cls_x = 3;
    P.cls_z = nz >= 2 ? 3 : 1;
    P.rot3 = (flags & SPECT_PLAN_ROTATION_3PASS) != 0;
    if (P.separable && !(flags & SPECT_PLAN_LOW_MEMORY)) {
        P.bucket = spect::fused_bucket(g, (size_t)smem_optin, &P.fused_nT);
        P.fast = P.bucket > 0;
    } else if (!(flags & SPECT_PLAN_LOW_MEMORY)) {
        P.bucket = spect::fused_dir_bucket(g, (size_t)smem_optin);
        P.fast = P.bucket > 0;
        P.fused_nT = 1;
    }
    P.recompute = (flags & SPECT_PLAN_RECOMPUTE_ATTENUATION) != 0 && P.fast && !P.rot3;
    *bytes = plan_bytes_bound(P);
    return SPECT_OK;
}

spect_status spect_plan_create(spect_plan* out, int nx, int ny, int nz, int nview, const float* mu, float dy,
                               const float* psf, const float* psf_fx, const float* psf_fz, int px, int pz,
                               int nview_psf, const double* angles, unsigned flags, spect_stream stream)
{
    if (!out) return fail(SPECT_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx != ny) return fail(SPECT_EINVAL, "nx must equal ny (rotation in the x-y plane)");
    if (nx < 2 || nx > 1024) return fail(SPECT_EINVAL, "nx must be in [2, 1024]");
    if (nz < 1 || nz > 4096) return fail(SPECT_EINVAL, "nz must be in [1, 4096]");
    if (nview < 1 || nview > 4096) return fail(SPECT_EINVAL, "nview must be in [1, 4096]");
    if (px < 1 || pz < 1 || px > 127 || pz > 127 || (px % 2) == 0 || (pz % 2) == 0)
        return fail(SPECT_EINVAL, "PSF sizes px, pz must be odd and in [1, 127]");
    if (nview_psf != 1 && nview_psf != nview) return fail(SPECT_EINVAL, "nview_psf must be 1 or nview");
    if (!(dy >= 0.f) || !isfinite(dy)) return fail(SPECT_EINVAL, "dy must be finite and >= 0");
    if ((psf_fx == nullptr) != (psf_fz == nullptr)) return fail(SPECT_EINVAL, "give both psf_fx and psf_fz or neither");
    if (!psf && !psf_fx) return fail(SPECT_EINVAL, "no PSF given (psf or psf_fx/psf_fz)");
    if ((flags & ~(unsigned)(SPECT_PLAN_PREFER_SEPARABLE | SPECT_PLAN_LOW_MEMORY | SPECT_PLAN_ROTATION_3PASS |
                             SPECT_PLAN_RECOMPUTE_ATTENUATION)) != 0)
        return fail(SPECT_EINVAL, "unknown flag bits");
    const void* ins[] = {mu, psf, psf_fx, psf_fz};
    for (const void* p : ins)
        if (p && !aligned16(p)) return fail(SPECT_EINVAL, "device inputs must be 16-byte aligned");
    if ((size_t)nview * nx * ny * 6 >= (size_t)INT32_MAX) return fail(SPECT_EUNSUPPORTED, "nview*nx*ny too large");
    if ((size_t)nx * ny * nz >= (size_t)INT32_MAX / 2) return fail(SPECT_EUNSUPPORTED, "nx*ny*nz too large");
    if (angles)
        for (int l = 0; l < nview; ++l)
            if (!isfinite(angles[l])) return fail(SPECT_EINVAL, "angles must be finite");

    cudaStream_t st = (cudaStream_t)stream;
    spect_plan_s* P = new spect_plan_s();
    P->home = st;
    Geometry& g = P->g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.nview = nview;
    g.px = px; g.pz = pz; g.nvp = nview_psf;
    g.cint = (nx - 1) / 2;
    g.cfrac = (nx - 1) % 2 ? 0.5f : 0.f;
    g.dy = dy;
    g.has_mu = mu != nullptr;
    P->separable = psf_fx && (!psf || (flags & SPECT_PLAN_PREFER_SEPARABLE));
    P->ps = (nx * nz + 3) & ~3;
    P->ts = (5 * nx + 3) & ~3;
    P->cls_x = 3;
    P->cls_z = nz >= 2 ? 3 : 1;

    int dev = 0, smem_optin = 0;
    spect_status r = SPECT_OK;
#define PLAN_TRY(expr, what)                                                                  \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            free_plan(P);                                                                     \
            return fail(SPECT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_));     \
        }                                                                                     \
    } while (0)
#define PLAN_ALLOC(ptr, n, what)                           \
    do {                                                   \
        r = dalloc(P, &(ptr), (n), what);                  \
        if (r != SPECT_OK) {                               \
            std::string m_ = g_err;                        \
            free_plan(P);                                  \
            return fail(r, m_);                            \
        }                                                  \
    } while (0)

    PLAN_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    PLAN_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "device query");
    P->smem_optin = smem_optin;
    {
        int pools = 0;
        PLAN_TRY(cudaDeviceGetAttribute(&pools, cudaDevAttrMemoryPoolsSupported, dev), "device query");
        P->pooled = pools != 0;
    }
    if (P->separable && !(flags & SPECT_PLAN_LOW_MEMORY)) {
        P->bucket = spect::fused_bucket(g, (size_t)smem_optin, &P->fused_nT);
        P->fast = P->bucket > 0;
    } else if (!(flags & SPECT_PLAN_LOW_MEMORY)) {
        // full PSF: the fused full-PSF blur kernels, untiled planes only
        P->bucket = spect::fused_dir_bucket(g, (size_t)smem_optin);
        P->fast = P->bucket > 0;
        P->fused_nT = 1;
    }
    P->rot3 = (flags & SPECT_PLAN_ROTATION_3PASS) != 0;
    if (P->rot3 && !P->fast) {
        free_plan(P);
        return fail(SPECT_EUNSUPPORTED, "the three-pass rotation runs on the fused kernels (not a low-memory plan)");
    }
    P->recompute = (flags & SPECT_PLAN_RECOMPUTE_ATTENUATION) != 0;
    if (P->recompute && (!P->fast || P->rot3)) {
        free_plan(P);
        return fail(SPECT_EUNSUPPORTED,
                    "recomputed attenuation runs on the fused kernels with the bilinear rotation (not with a "
                    "low-memory plan, the three-pass rotation, or a geometry the fused kernels do not fit)");
    }
    if (P->separable) {
        P->sep_tk = spect::choose_sep_tile(g, P->cls_z, (size_t)smem_optin);
        if (P->sep_tk < 1) {
            free_plan(P);
            return fail(SPECT_EUNSUPPORTED, "separable PSF tile does not fit shared memory for this nx, pz");
        }
    } else if (!spect::direct_fits(g, (size_t)smem_optin)) {
        free_plan(P);
        return fail(SPECT_EUNSUPPORTED, "full PSF tile does not fit shared memory");
    }

    const size_t vol = (size_t)nx * ny * nz, nproj = (size_t)nx * nz * nview;
    const size_t nxy = (size_t)nx * ny, nrows = (size_t)nview_psf * ny;

    PLAN_ALLOC(P->err, 1, "error word");
    PLAN_TRY(cudaMemsetAsync(P->err, 0, sizeof(int), st), "clear error word");
    // attenuation map (zeros are never read when mu == NULL)
    PLAN_ALLOC(P->mu, vol, "mu");
    if (mu) PLAN_TRY(cudaMemcpyAsync(P->mu, mu, vol * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy mu");
    else PLAN_TRY(cudaMemsetAsync(P->mu, 0, vol * sizeof(float), st), "clear mu");

    // PSF and its edge-class variants for A'
    if (P->separable) {
        PLAN_ALLOC(P->fx, (size_t)px * nrows, "psf_fx");
        PLAN_ALLOC(P->fz, (size_t)pz * nrows, "psf_fz");
        PLAN_ALLOC(P->fx_adj, (size_t)3 * px * nrows, "psf_fx variants");
        PLAN_ALLOC(P->fz_adj, (size_t)P->cls_z * pz * nrows, "psf_fz variants");
        PLAN_TRY(cudaMemcpyAsync(P->fx, psf_fx, (size_t)px * nrows * sizeof(float), cudaMemcpyDeviceToDevice, st),
                 "copy psf_fx");
        PLAN_TRY(cudaMemcpyAsync(P->fz, psf_fz, (size_t)pz * nrows * sizeof(float), cudaMemcpyDeviceToDevice, st),
                 "copy psf_fz");
        PLAN_TRY(spect::launch_psf_variants(*P, nullptr, st), "PSF variant launch");
    } else {
        const size_t n = (size_t)px * pz * nrows;
        PLAN_ALLOC(P->psf, n, "psf");
        PLAN_ALLOC(P->psf_adj, n * P->cls_x * P->cls_z, "psf variants");
        PLAN_TRY(cudaMemcpyAsync(P->psf, psf, n * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy psf");
        float* scratch = nullptr;
        PLAN_TRY(raw_alloc(P, (void**)&scratch, n * P->cls_x * sizeof(float), st), "PSF variant scratch");
        cudaError_t e1 = spect::launch_psf_variants(*P, scratch, st);
        raw_free(P, scratch, st);
        cudaError_t e2 = cudaStreamSynchronize(st);
        PLAN_TRY(e1, "PSF variant launch");
        PLAN_TRY(e2, "PSF variant build");
    }

    // per-view rotation constants
    {
        std::vector<ViewRot> vr(nview);
        spect::make_view_rot(nx, nview, angles, vr.data());
        PLAN_ALLOC(P->rot, (size_t)nview, "rotation constants");
        PLAN_TRY(cudaMemcpyAsync(P->rot, vr.data(), nview * sizeof(ViewRot), cudaMemcpyHostToDevice, st),
                 "upload rotation constants");
        PLAN_TRY(cudaStreamSynchronize(st), "rotation constants");
    }

    // adjacency lists of the transposed rotation (count, scan on host, fill)
    {
        const size_t nlist = nxy * nview;
        int* d_counts = nullptr;
        int* d_max = nullptr;
        PLAN_TRY(raw_alloc(P, (void**)&d_counts, nlist * sizeof(int), st), "adjacency counts");
        PLAN_TRY(raw_alloc(P, (void**)&d_max, sizeof(int), st), "adjacency max");
        cudaMemsetAsync(d_max, 0, sizeof(int), st);
        cudaError_t e1 = spect::launch_build_adjacency(*P, 0, d_counts, d_max, st);
        std::vector<int> counts(nlist);
        int mx = 0;
        cudaError_t e2 = cudaMemcpyAsync(counts.data(), d_counts, nlist * sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaError_t e3 = cudaMemcpyAsync(&mx, d_max, sizeof(int), cudaMemcpyDeviceToHost, st);
        raw_free(P, d_counts, st);
        raw_free(P, d_max, st);
        cudaError_t e4 = cudaStreamSynchronize(st);
        PLAN_TRY(e1, "adjacency count launch");
        PLAN_TRY(e2, "adjacency counts download");
        PLAN_TRY(e3, "adjacency max download");
        PLAN_TRY(e4, "adjacency count");
        if (P->rot3) mx = std::max(mx, 8);  // eight entries per (voxel, view) for the three-pass lists
        P->adj_max = mx;
        if (P->fast && mx > 8) P->fast = 0;  // fixed-length lists are instantiated up to 8 entries
        if (P->fast) {
            PLAN_ALLOC(P->adjf, nlist * (size_t)std::max(mx, 1), "adjacency lists");
            if (mx < 1) P->adj_max = 1;
            PLAN_TRY(spect::launch_build_adjacency_fixed(*P, st), "adjacency fill launch");
        } else {
            std::vector<int> off(nlist + 1);
            size_t tot = 0;
            for (size_t m = 0; m < nlist; ++m) {
                off[m] = (int)tot;
                tot += (size_t)counts[m];
            }
            off[nlist] = (int)tot;
            PLAN_ALLOC(P->adj_off, nlist + 1, "adjacency offsets");
            PLAN_ALLOC(P->adj, std::max<size_t>(tot, 1), "adjacency entries");
            PLAN_TRY(cudaMemcpyAsync(P->adj_off, off.data(), (nlist + 1) * sizeof(int), cudaMemcpyHostToDevice, st),
                     "upload adjacency offsets");
            PLAN_TRY(spect::launch_build_adjacency(*P, 1, nullptr, nullptr, st), "adjacency fill launch");
        }
        PLAN_TRY(cudaStreamSynchronize(st), "adjacency fill");
    }

    // work slab and EM buffers
    const size_t budget = P->recompute ? recompute_budget_bytes() : slab_budget_bytes(P->fast);
    // the fused path stores padded planes (rotated image planes or adjoint planes)
    const size_t per_view = std::max(vol, P->fast ? spect::fused_slab_per_view(*P) : vol);
    P->chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)nview, budget / (view_bytes(*P, per_view))));
    PLAN_ALLOC(P->slab, per_view * (size_t)P->chunk, "work slab");
    P->slab_cap = per_view * (size_t)P->chunk;
    // fused adjoint: all views of the slab in one pass by default (measured
    // faster than L2-sized passes); SPECT_ADJ_CHUNK sets fewer views per pass,
    // with a depth-group size that keeps about two blocks per SM (tuning)
    P->adj_chunk = P->chunk;
    P->adj_J = 8;
    if (const char* env = getenv("SPECT_ADJ_CHUNK")) {
        if (atoi(env) > 0) {
            P->adj_chunk_req = atoi(env);
            P->adj_chunk = std::min(std::min(atoi(env), nview), P->chunk);
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int want_groups = std::max(1, (2 * std::max(sms, 1) + P->adj_chunk - 1) / P->adj_chunk);
            P->adj_J = std::max(1, std::min(8, (ny + want_groups - 1) / want_groups));
        }
    }
    PLAN_ALLOC(P->e, vol, "EM accumulator");
    PLAN_ALLOC(P->ratio, nproj, "EM ratio");
    PLAN_ALLOC(P->s, vol, "sensitivity");

    // fused path: attenuation cache for every view (or for one view chunk,
    // recomputed per chunk), internal-layout buffers
    if (P->fast) {
        const int mu_views = P->recompute ? P->chunk : nview;
        PLAN_ALLOC(P->mubar, (size_t)ny * P->ps * mu_views, "attenuation cache");
        P->mubar_cap = (size_t)ny * P->ps * mu_views;
        PLAN_ALLOC(P->xt, vol, "internal image");
        PLAN_ALLOC(P->et, vol, "internal back-projection");
        PLAN_ALLOC(P->st, vol, "internal sensitivity");
        PLAN_ALLOC(P->ut, vol, "internal regulariser target");
        PLAN_ALLOC(P->part, nproj * (size_t)spect::fused_groups(*P), "depth-group partial sums");
        P->part_cap = nproj * (size_t)spect::fused_groups(*P);
        // mu in the [j][i][k] layout (temporary, the slab serves as scratch)
        PLAN_TRY(spect::launch_transpose(P->mu, P->slab, nz, (int)nxy, st), "mu transpose launch");
        if (P->rot3) {
            // three passes: the eight-tap table of the forward rotation kernel, the
            // eight-entry lists of the adjoint gather (in adjf), and the attenuation
            // cache from mu turned the same way (one volume of scratch)
            PLAN_ALLOC(P->r3_tab, (size_t)nview * ny * spect::rot3_ts8(nx), "three-pass table");
            float* scratch = nullptr;
            PLAN_TRY(raw_alloc(P, (void**)&scratch, vol * sizeof(float), st), "three-pass scratch");
            cudaError_t e3 = spect::build_rot3(*P, angles, P->slab, scratch, st);
            raw_free(P, scratch, st);
            PLAN_TRY(e3, "three-pass rotation set-up");
            PLAN_TRY(spect::build_gather(*P, st), "patch gather set-up");  // boxes of the three-pass lists
            drop_fixed_lists(P, st);
        } else if (P->recompute) {
            // mu stays in the [j][i][k] layout; the factors are made per view chunk
            PLAN_ALLOC(P->mut, vol, "attenuation map (internal layout)");
            PLAN_TRY(cudaMemcpyAsync(P->mut, P->slab, vol * sizeof(float), cudaMemcpyDeviceToDevice, st),
                     "attenuation map copy");
            PLAN_ALLOC(P->rtab, (size_t)nview * ny * P->ts, "rotation tables");
            PLAN_TRY(spect::launch_rot_tables(*P, st), "rotation table launch");
            PLAN_TRY(spect::build_gather(*P, st), "patch gather set-up");
            drop_fixed_lists(P, st);
        } else {
            PLAN_ALLOC(P->rtab, (size_t)nview * ny * P->ts, "rotation tables");
            PLAN_TRY(spect::launch_rot_tables(*P, st), "rotation table launch");
            PLAN_TRY(spect::launch_mubar_cache(*P, P->slab, st), "attenuation cache launch");
            PLAN_TRY(spect::build_gather(*P, st), "patch gather set-up");
            drop_fixed_lists(P, st);
            PLAN_TRY(spect::build_rotpatch(*P, st), "patch rotation set-up");
        }
    }
    PLAN_TRY(cudaStreamSynchronize(st), "plan set-up");
    *out = P;
    return SPECT_OK;
#undef PLAN_TRY
#undef PLAN_ALLOC
}

spect_status spect_plan_destroy(spect_plan P)
{
    if (!P) return SPECT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    // the device is idle: free on the legacy default stream and wait, so the
    // memory is back in the pool when this returns
    free_plan(P, (cudaStream_t)0);
    cudaError_t e2 = cudaStreamSynchronize((cudaStream_t)0);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(SPECT_ECUDA, std::string("synchronise before destroy: ") + cudaGetErrorString(e));
    return SPECT_OK;
}

spect_status spect_plan_release(spect_plan P, spect_stream stream)
{
    if (!P) return SPECT_OK;
    free_plan(P, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SPECT_ECUDA, std::string("stream-ordered release: ") + cudaGetErrorString(e));
    return SPECT_OK;
}

spect_status spect_forward(spect_plan P, const float* x, float* v, spect_stream stream)
{
    spect_status r = check_call(P, x, v, "x", "v");
    if (r != SPECT_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    if (P->fast) {
        r = to_internal(P, x, P->xt, st);
        if (r != SPECT_OK) return r;
        return fast_forward(P, P->xt, v, nullptr, nullptr, st);
    }
    return run_forward(P, x, v, nullptr, nullptr, st);
}

spect_status spect_back(spect_plan P, const float* v, float* x, spect_stream stream)
{
    spect_status r = check_call(P, v, x, "v", "x");
    if (r != SPECT_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    if (P->fast) {
        r = fast_back(P, v, P->et, spect::EmArgs(), st);
        if (r != SPECT_OK) return r;
        return from_internal(P, P->et, x, st);
    }
    return run_back(P, v, x, spect::EmArgs(), st);
}

spect_status spect_sensitivity(spect_plan P, float* s, spect_stream stream)
{
    spect_status r = check_call(P, s, s, "s", "s");
    if (r != SPECT_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    r = ensure_sensitivity(P, st);
    if (r != SPECT_OK) return r;
    const size_t vol = (size_t)P->g.nx * P->g.ny * P->g.nz;
    SPECT_CUDA_TRY(cudaMemcpyAsync(s, P->s, vol * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy sensitivity");
    return SPECT_OK;
}

spect_status spect_em_step(spect_plan P, float* x, const float* y, const float* rbar, int niter, spect_stream stream)
{
    return spect_em_step_reg(P, x, y, rbar, nullptr, 0.f, niter, stream);
}

spect_status spect_em_step_reg(spect_plan P, float* x, const float* y, const float* rbar, const float* u, float beta,
                               int niter, spect_stream stream)
{
    spect_status r = check_call(P, x, y, "x", "y");
    if (r != SPECT_OK) return r;
    if (rbar && !aligned16(rbar)) return fail(SPECT_EINVAL, "rbar is not 16-byte aligned");
    if (niter < 0) return fail(SPECT_EINVAL, "niter must be >= 0");
    if (!(beta >= 0.f) || !isfinite(beta)) return fail(SPECT_EINVAL, "beta must be finite and >= 0");
    if (beta > 0.f && !u) return fail(SPECT_EINVAL, "u is required when beta > 0");
    if (u && !aligned16(u)) return fail(SPECT_EINVAL, "u is not 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    r = ensure_sensitivity(P, st);
    if (r != SPECT_OK) return r;
    return em_iterate(P, x, y, rbar, u, beta, niter, st);
}

}  // extern "C"

namespace {

// niter EM updates of x (Eqs. (7)-(8)) once the sensitivity is cached:
// everything stream-ordered on st, no host synchronisation (capturable).
spect_status em_iterate(spect_plan_s* P, float* x, const float* y, const float* rbar, const float* u, float beta,
                        int niter, cudaStream_t st)
{
    spect_status r = SPECT_OK;
    if (niter == 0) return SPECT_OK;
    spect::EmArgs em;
    em.beta = beta > 0.f ? beta : 0.f;
    if (P->fast) {
        r = to_internal(P, x, P->xt, st);
        if (r != SPECT_OK) return r;
        if (em.beta > 0.f) {
            r = to_internal(P, u, P->ut, st);
            if (r != SPECT_OK) return r;
            em.u = P->ut;
        }
        em.x = P->xt;
        em.s = P->st;
        for (int it = 0; it < niter; ++it) {
            r = fast_forward(P, P->xt, P->ratio, y, rbar, st);
            if (r != SPECT_OK) return r;
            r = fast_back(P, P->ratio, P->et, em, st);
            if (r != SPECT_OK) return r;
        }
        return from_internal(P, P->xt, x, st);
    }
    em.x = x;
    em.s = P->s;
    em.u = em.beta > 0.f ? u : nullptr;
    for (int it = 0; it < niter; ++it) {
        r = run_forward(P, x, P->ratio, y, rbar, st);
        if (r != SPECT_OK) return r;
        r = run_back(P, P->ratio, P->e, em, st);
        if (r != SPECT_OK) return r;
    }
    return SPECT_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// One thread waits, with the bounded mbarrier wait of the fused kernels but a
// limit of `spin_clocks`, on a barrier that nothing ever completes; the wait
// runs out and the block records SPECT_ETIMEOUT in the error word, exactly as a
// fused kernel whose bulk copy never landed would.
__global__ void k_wait_selftest(int* err, long long spin_clocks)
{
    __shared__ __align__(8) uint64_t bar;
    spect::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bool done = spect::mbar_try_wait(&bar, 0u);
    const long long t0 = clock64();
    while (!done && clock64() - t0 < spin_clocks) done = spect::mbar_try_wait(&bar, 0u);
    if (!done && err) atomicExch(err, (int)SPECT_ETIMEOUT);
}

}  // namespace

extern "C" {

spect_status spect_plan_selftest_timeout(spect_plan P, long long spin_clocks, spect_stream stream)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    if (spin_clocks < 0 || spin_clocks > (1ll << 31)) return fail(SPECT_EINVAL, "spin_clocks must be in [0, 2^31]");
    k_wait_selftest<<<1, 1, 0, (cudaStream_t)stream>>>(P->err, spin_clocks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SPECT_ECUDA, std::string("self-test launch: ") + cudaGetErrorString(e));
    return SPECT_OK;
}

spect_status spect_plan_check_stream(spect_plan P, spect_stream stream)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, P->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && h != 0) e = cudaMemsetAsync(P->err, 0, sizeof(int), st);
    if (e != cudaSuccess) return fail(SPECT_ECUDA, std::string("reading the plan's error word: ") + cudaGetErrorString(e));
    if (h == SPECT_ETIMEOUT) return fail(SPECT_ETIMEOUT, "a bounded wait on a bulk copy ran out; outputs are invalid");
    if (h != 0) return fail(SPECT_ECUDA, "device error word set");
    return SPECT_OK;
}

spect_status spect_plan_check(spect_plan P)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    int h = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, P->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h != 0) e = cudaMemset(P->err, 0, sizeof(int));
    if (e != cudaSuccess) return fail(SPECT_ECUDA, std::string("reading the plan's error word: ") + cudaGetErrorString(e));
    if (h == SPECT_ETIMEOUT) return fail(SPECT_ETIMEOUT, "a bounded wait on a bulk copy ran out; outputs are invalid");
    if (h != 0) return fail(SPECT_ECUDA, "device error word set");
    return SPECT_OK;
}

spect_status spect_profile_enable(spect_plan P, int enable)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    P->prof = enable != 0;
    return SPECT_OK;
}

spect_status spect_profile_read(spect_plan P, long long* launches, double* ms, int reset)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    cudaError_t e = drain_profile(P);
    for (int k = 0; k < SPECT_K_COUNT; ++k) {
        if (launches) launches[k] = P->launches[k];
        if (ms) ms[k] = P->prof_ms[k];
        if (reset) {
            P->launches[k] = 0;
            P->prof_ms[k] = 0.0;
        }
    }
    if (e != cudaSuccess) return fail(SPECT_ECUDA, std::string("reading kernel timings: ") + cudaGetErrorString(e));
    return SPECT_OK;
}

spect_status spect_plan_info(spect_plan P, int* separable, int* fused, int* view_chunk, size_t* device_bytes)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    if (separable) *separable = P->separable;
    if (fused) *fused = P->fast;
    if (view_chunk) *view_chunk = P->chunk;
    if (device_bytes) *device_bytes = P->bytes;
    return SPECT_OK;
}

}  // extern "C"

// ============================================================================
// Tuning of the fused kernels' launch shapes, the autotuner, and batches of
// plans run as one CUDA graph (the paper has no counterpart for any of these).
// ============================================================================
struct spect_batch_s {
    std::vector<spect_plan_s*> plans;
    std::vector<cudaStream_t> side;  // one capture branch per plan (round-robin when plans outnumber them)
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t origin = nullptr;   // the capture's origin stream (the caller's may be the legacy stream)
    // the instantiated graph and the arguments it was captured with
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;
    long long graph_launches = 0;   // kernels per graph launch
    // grouped launches (every plan on the fused separable path): the plans split
    // into a few branches of about equal work; on each branch one launch per
    // stage and kernel variant over the branch's plans
    std::vector<spect::GroupedBatch> grouped;
    int grouped_on = 0;
    int grouped_branches = 0;  // spect_batch_set_grouped: 0 = a graph branch per plan
};

namespace {

spect_status realloc_floats(spect_plan_s* P, float** p, size_t* cap, size_t need, cudaStream_t st, const char* what)
{
    if (need <= *cap) return SPECT_OK;
    float* q = nullptr;
    cudaError_t e = raw_alloc(P, (void**)&q, need * sizeof(float), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SPECT_ENOMEM : SPECT_ECUDA,
                    std::string("allocating ") + what + ": " + cudaGetErrorString(e));
    }
    if (((uintptr_t)q & 255) != 0) {
        raw_free(P, q, st);
        return fail(SPECT_ECUDA, std::string("allocation of ") + what + " is not 256-byte aligned");
    }
    raw_free(P, *p, st);
    P->bytes += (need - *cap) * sizeof(float);
    *p = q;
    *cap = need;
    return SPECT_OK;
}

// Set the fused kernels' depth-group sizes and column-tile count, growing the
// work slab and the partial-sum buffer when the new shape needs more room.
spect_status reconfigure(spect_plan_s* P, int J, int adj_J, int tiles, cudaStream_t st)
{
    if (!P->fast) return fail(SPECT_EUNSUPPORTED, "launch-shape tuning applies to the fused kernels only");
    const Geometry& g = P->g;
    if (J < 1 || J > 32 || adj_J < 1 || adj_J > 32 || tiles < 1)
        return fail(SPECT_EINVAL, "fused_J and adj_J must be in [1, 32], tiles >= 1");
    int dev = 0, smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(SPECT_ECUDA, "device query failed");
    }
    const int nt = P->separable ? spect::fused_tiles_fit(g, P->bucket, J, adj_J, tiles, (size_t)smem)
                                : (tiles == 1 && spect::fused_dir_fit(g, P->bucket, J, adj_J, (size_t)smem) ? 1 : 0);
    if (nt == 0) return fail(SPECT_EUNSUPPORTED, "this launch shape does not fit shared memory");
    const int oJ = P->fused_J, oaJ = P->adj_J, ont = P->fused_nT;
    P->fused_J = J;
    P->adj_J = adj_J;
    P->fused_nT = nt;
    const size_t vol = (size_t)g.nx * g.ny * g.nz, nproj = (size_t)g.nx * g.nz * g.nview;
    const size_t per_view = std::max(vol, spect::fused_slab_per_view(*P));
    const size_t budget = P->recompute ? recompute_budget_bytes() : slab_budget_bytes(true);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)g.nview, budget / view_bytes(*P, per_view)));
    spect_status r = realloc_floats(P, &P->slab, &P->slab_cap, per_view * (size_t)chunk, st, "work slab");
    if (r == SPECT_OK)
        r = realloc_floats(P, &P->part, &P->part_cap, nproj * (size_t)spect::fused_groups(*P), st,
                           "depth-group partial sums");
    if (r == SPECT_OK && P->recompute)  // the attenuation factors of one chunk
        r = realloc_floats(P, &P->mubar, &P->mubar_cap, (size_t)g.ny * P->ps * chunk, st, "attenuation factors");
    if (r != SPECT_OK) {
        P->fused_J = oJ;
        P->adj_J = oaJ;
        P->fused_nT = ont;
        return r;
    }
    P->chunk = chunk;
    P->adj_chunk = P->adj_chunk_req > 0 ? std::min(P->adj_chunk_req, chunk) : chunk;
    return SPECT_OK;
}

// One pass over every view, as the grouped batch launches need: grow the work
// slab (stream-ordered on st) so it holds every view of a fused separable plan.
spect_status single_pass(spect_plan_s* P, cudaStream_t st)
{
    if (!P->fast || !P->separable || P->rot3 || P->recompute) return SPECT_OK;
    const Geometry& g = P->g;
    if (P->chunk >= g.nview && P->adj_chunk >= g.nview) return SPECT_OK;
    if (P->adj_chunk_req > 0 && P->adj_chunk_req < g.nview) return SPECT_OK;  // adjoint passes asked for
    const size_t vol = (size_t)g.nx * g.ny * g.nz;
    const size_t per_view = std::max(vol, spect::fused_slab_per_view(*P));
    spect_status r = realloc_floats(P, &P->slab, &P->slab_cap, per_view * (size_t)g.nview, st, "work slab");
    if (r != SPECT_OK) return r;
    P->chunk = g.nview;
    P->adj_chunk = g.nview;
    return SPECT_OK;
}

// Device time of one call of fn (best of `reps` after one warm-up run).
template <class F>
spect_status time_best(cudaStream_t st, int reps, float* best, F&& fn)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        cudaGetLastError();
        return fail(SPECT_ECUDA, "event creation failed");
    }
    spect_status r = fn();
    *best = 1e30f;
    for (int k = 0; k < reps && r == SPECT_OK; ++k) {
        cudaEventRecord(a, st);
        r = fn();
        cudaEventRecord(b, st);
        float ms = 0.f;
        if (r == SPECT_OK && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
            *best = std::min(*best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaError_t e = cudaGetLastError();
    if (r == SPECT_OK && e != cudaSuccess) r = fail(SPECT_ECUDA, std::string("timing: ") + cudaGetErrorString(e));
    return r;
}

struct Tuned {
    int J, adj_J, tiles, rotpatch;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int, int>, Tuned> g_tuned;  // per geometry, mode and device

}  // namespace

extern "C" {

spect_status spect_plan_set_tuning(spect_plan P, int fused_J, int adj_J, int tiles, spect_stream stream)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    return reconfigure(P, fused_J, adj_J, tiles, (cudaStream_t)stream);
}

spect_status spect_plan_get_tuning(spect_plan P, int* fused_J, int* adj_J, int* tiles)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    if (fused_J) *fused_J = P->fused_J;
    if (adj_J) *adj_J = P->adj_J;
    if (tiles) *tiles = P->fused_nT;
    return SPECT_OK;
}

spect_status spect_plan_autotune(spect_plan P, spect_stream stream)
{
    if (!P) return fail(SPECT_EINVAL, "plan is NULL");
    if (!P->fast) return SPECT_OK;  // the low-memory kernels have no launch shape to choose
    cudaStream_t st = (cudaStream_t)stream;
    const Geometry& g = P->g;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, g.nx, g.nz, g.nview, g.nvp, P->bucket, (int)P->g.has_mu, P->recompute);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            P->rotpatch_on = P->rotpatch && it->second.rotpatch;
            return reconfigure(P, it->second.J, it->second.adj_J, it->second.tiles, st);
        }
    }
    // inputs of the timed calls: the plan's own scratch (x_t = 1, v = 1)
    const size_t vol = (size_t)g.nx * g.ny * g.nz, nproj = (size_t)g.nx * g.nz * g.nview;
    if (spect::launch_fill(P->xt, vol, 1.f, st) != cudaSuccess ||
        spect::launch_fill(P->ratio, nproj, 1.f, st) != cudaSuccess)
        return fail(SPECT_ECUDA, "fill launch failed");
    const int prof = P->prof;
    P->prof = 0;
    const int base = P->fused_nT;
    const int nib = (g.nx + 15) / 16;
    std::vector<int> tile_cands;
    for (int t : {base, base + 1, 2 * base, 4 * base})
        if (t <= nib && std::find(tile_cands.begin(), tile_cands.end(), t) == tile_cands.end()) tile_cands.push_back(t);
    if (!P->separable) tile_cands.assign(1, 1);  // the full-PSF kernels run untiled
    std::vector<int> Js;
    for (int J : {4, 8, 12, 16, 20, 24, 32})
        if (J <= std::max(g.ny, 4)) Js.push_back(J);
    Tuned best{P->fused_J, P->adj_J, base, 0};
    P->rotpatch_on = 0;
    float best_ms = 1e30f;
    spect_status r = SPECT_OK;
    for (int t : tile_cands) {
        float fbest = 1e30f, abest = 1e30f;
        int fJ = 0, aJ = 0;
        for (int J : Js) {
            if (reconfigure(P, J, Js.front(), t, st) != SPECT_OK) continue;
            float ms = 0.f;
            r = time_best(st, 3, &ms, [&] { return fast_forward(P, P->xt, P->ratio, nullptr, nullptr, st); });
            if (r != SPECT_OK) break;
            if (ms < fbest) fbest = ms, fJ = J;
        }
        if (r != SPECT_OK) break;
        for (int J : Js) {
            if (!fJ || reconfigure(P, fJ, J, t, st) != SPECT_OK) continue;
            float ms = 0.f;
            r = time_best(st, 3, &ms, [&] { return fast_back(P, P->ratio, P->et, spect::EmArgs(), st); });
            if (r != SPECT_OK) break;
            if (ms < abest) abest = ms, aJ = J;
        }
        if (r != SPECT_OK) break;
        if (fJ && aJ && fbest + abest < best_ms) {
            best_ms = fbest + abest;
            best = {fJ, aJ, t, 0};
        }
    }
    if (r == SPECT_OK) r = reconfigure(P, best.J, best.adj_J, best.tiles, st);
    // the rotation kernel: plane gathers or patch-staged boxes (untiled planes only)
    if (r == SPECT_OK && P->rotpatch && P->fused_nT == 1) {
        float ms_plane = 0.f, ms_patch = 0.f;
        r = time_best(st, 3, &ms_plane, [&] { return fast_forward(P, P->xt, P->ratio, nullptr, nullptr, st); });
        P->rotpatch_on = 1;
        if (r == SPECT_OK)
            r = time_best(st, 3, &ms_patch, [&] { return fast_forward(P, P->xt, P->ratio, nullptr, nullptr, st); });
        P->rotpatch_on = r == SPECT_OK && ms_patch < ms_plane;
        best.rotpatch = P->rotpatch_on;
    }
    P->prof = prof;
    if (r != SPECT_OK) return r;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
    return SPECT_OK;
}

spect_status spect_batch_create(spect_batch* out, const spect_plan* plans, int n)
{
    if (!out) return fail(SPECT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!plans || n < 1) return fail(SPECT_EINVAL, "need at least one plan");
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return fail(SPECT_EINVAL, "plan is NULL");
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return fail(SPECT_EINVAL, "a plan appears twice in the batch");
    }
    spect_batch_s* B = new spect_batch_s();
    B->plans.assign(plans, plans + n);
    const int ns = std::min(n, 32);
    cudaError_t e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->origin, cudaStreamNonBlocking);
    for (int i = 0; i < ns && e == cudaSuccess; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t j = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) B->side.push_back(s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (e == cudaSuccess) B->join.push_back(j);
    }
    if (e != cudaSuccess) {
        spect_batch_destroy(B);
        cudaGetLastError();
        return fail(SPECT_ECUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
    }
    *out = B;
    return SPECT_OK;
}

spect_status spect_batch_em_step(spect_batch B, float* const* x, const float* const* y, const float* const* rbar,
                                 int niter, spect_stream stream)
{
    if (!B) return fail(SPECT_EINVAL, "batch is NULL");
    if (!x || !y) return fail(SPECT_EINVAL, "x and y pointer arrays are required");
    if (niter < 0) return fail(SPECT_EINVAL, "niter must be >= 0");
    const int n = (int)B->plans.size();
    for (int i = 0; i < n; ++i) {
        spect_status r = check_call(B->plans[i], x[i], y[i], "x", "y");
        if (r != SPECT_OK) return r;
        if (rbar && rbar[i] && !aligned16(rbar[i])) return fail(SPECT_EINVAL, "rbar is not 16-byte aligned");
    }
    cudaStream_t st = (cudaStream_t)stream;
    // sensitivities are computed outside the graph (once per plan)
    for (spect_plan_s* P : B->plans) {
        spect_status r = ensure_sensitivity(P, st);
        if (r != SPECT_OK) return r;
    }
    if (niter == 0) return SPECT_OK;
    std::vector<const void*> key;
    key.push_back((const void*)(intptr_t)niter);
    for (int i = 0; i < n; ++i) {
        key.push_back(x[i]);
        key.push_back(y[i]);
        key.push_back(rbar ? rbar[i] : nullptr);
    }
    if (!B->exec || key != B->key) {
        if (B->exec) cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
        // grouped launches when every plan runs the fused separable kernels in one
        // pass (SPECT_BATCH_GROUPED=0, testing: a graph branch per plan instead)
        for (spect::GroupedBatch& gb : B->grouped) spect::free_grouped(gb);
        B->grouped.clear();
        B->grouped_on = 0;
        bool grp = B->grouped_branches > 0;
        for (spect_plan_s* P : B->plans) {
            if (!grp) break;
            if (single_pass(P, st) != SPECT_OK) {  // no room for every view: a graph branch per plan
                cudaGetLastError();
                grp = false;
            }
            grp = grp && spect::groupable(*P);
        }
        if (grp) {
            // branches: longest-processing-time assignment of the plans by work
            const int nbr = std::min(B->grouped_branches, std::min(n, (int)B->side.size()));
            std::vector<int> order(n);
            std::iota(order.begin(), order.end(), 0);
            auto work = [&](int i) {
                const Geometry& g = B->plans[i]->g;
                return (double)g.nx * g.ny * g.nz * g.nview;
            };
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
            std::vector<std::vector<int>> members(nbr);
            std::vector<double> load(nbr, 0.0);
            for (int i : order) {
                const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                members[b].push_back(i);
                load[b] += work(i);
            }
            B->grouped.resize(nbr);
            cudaError_t eg = cudaSuccess;
            for (int b = 0; b < nbr && eg == cudaSuccess; ++b) {
                std::vector<spect_plan_s*> pl;
                std::vector<float*> xb;
                std::vector<const float*> yb, rb;
                for (int i : members[b]) {
                    pl.push_back(B->plans[i]);
                    xb.push_back(x[i]);
                    yb.push_back(y[i]);
                    rb.push_back(rbar ? rbar[i] : nullptr);
                }
                eg = spect::build_grouped(pl, xb.data(), yb.data(), rb.data(), B->grouped[b]);
            }
            if (eg != cudaSuccess) {
                for (spect::GroupedBatch& gb : B->grouped) spect::free_grouped(gb);
                B->grouped.clear();
                cudaGetLastError();
                return fail(SPECT_ECUDA, std::string("grouped batch set-up: ") + cudaGetErrorString(eg));
            }
            B->grouped_on = 1;
        }
        std::vector<int> prof(n);
        std::vector<long long> before(n);
        for (int i = 0; i < n; ++i) {
            prof[i] = B->plans[i]->prof;
            B->plans[i]->prof = 0;  // no timing events inside the graph
            before[i] = 0;
            for (int k = 0; k < SPECT_K_COUNT; ++k) before[i] += B->plans[i]->launches[k];
        }
        // captured on the batch's own origin stream; launched on the caller's
        cudaStream_t cs = B->origin;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        spect_status r = e == cudaSuccess ? SPECT_OK : fail(SPECT_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        if (r == SPECT_OK) e = cudaEventRecord(B->fork, cs);
        const int ns = (int)B->side.size();
        for (int s = 0; s < ns && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(B->side[s], B->fork, 0);
        if (r == SPECT_OK && e != cudaSuccess) r = fail(SPECT_ECUDA, std::string("fork: ") + cudaGetErrorString(e));
        long long grouped_kernels = 0;
        if (B->grouped_on) {
            // one chain per branch: layouts in, niter x (rotation, blur, reduce +
            // ratio, blur adjoint, gather + update), layouts out
            for (size_t b = 0; b < B->grouped.size() && r == SPECT_OK; ++b) {
                cudaStream_t bs = B->side[b];
                auto run = [&](const std::vector<spect::GroupLaunch>& L) {
                    for (const spect::GroupLaunch& f : L) {
                        if (r != SPECT_OK) return;
                        const cudaError_t el = f(bs);
                        if (el != cudaSuccess)
                            r = fail(SPECT_ECUDA, std::string("grouped launch: ") + cudaGetErrorString(el));
                        ++grouped_kernels;
                    }
                };
                run(B->grouped[b].head);
                for (int it = 0; it < niter; ++it) run(B->grouped[b].iter);
                run(B->grouped[b].tail);
            }
        }
        for (int i = 0; i < n && r == SPECT_OK && !B->grouped_on; ++i)
            r = em_iterate(B->plans[i], x[i], y[i], rbar ? rbar[i] : nullptr, nullptr, 0.f, niter, B->side[i % ns]);
        for (int s = 0; s < ns && r == SPECT_OK; ++s) {
            e = cudaEventRecord(B->join[s], B->side[s]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, B->join[s], 0);
            if (e != cudaSuccess) r = fail(SPECT_ECUDA, std::string("join: ") + cudaGetErrorString(e));
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);  // always ends the capture
        if (r == SPECT_OK && e2 != cudaSuccess) r = fail(SPECT_ECUDA, std::string("end capture: ") + cudaGetErrorString(e2));
        if (r == SPECT_OK) {
            e = cudaGraphInstantiate(&B->exec, graph, 0);
            if (e != cudaSuccess) {
                B->exec = nullptr;
                r = fail(SPECT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            }
        }
        if (graph) cudaGraphDestroy(graph);
        long long total = 0;
        for (int i = 0; i < n; ++i) {
            B->plans[i]->prof = prof[i];
            long long now = 0;
            for (int k = 0; k < SPECT_K_COUNT; ++k) now += B->plans[i]->launches[k];
            total += now - before[i];
        }
        cudaGetLastError();
        if (r != SPECT_OK) return r;
        B->graph_launches = B->grouped_on ? grouped_kernels : total;
        B->key = key;
    }
    cudaError_t e = cudaGraphLaunch(B->exec, st);
    if (e != cudaSuccess) return fail(SPECT_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return SPECT_OK;
}

spect_status spect_batch_set_grouped(spect_batch B, int branches)
{
    if (!B) return fail(SPECT_EINVAL, "batch is NULL");
    if (branches < 0 || branches > 32) return fail(SPECT_EINVAL, "branches must be in [0, 32]");
    if (branches != B->grouped_branches) {
        B->grouped_branches = branches;
        B->key.clear();  // captured again on the next call
    }
    return SPECT_OK;
}

spect_status spect_batch_info(spect_batch B, int* n_plans, long long* kernels_per_launch)
{
    if (!B) return fail(SPECT_EINVAL, "batch is NULL");
    if (n_plans) *n_plans = (int)B->plans.size();
    if (kernels_per_launch) *kernels_per_launch = B->graph_launches;
    return SPECT_OK;
}

spect_status spect_batch_destroy(spect_batch B)
{
    if (!B) return SPECT_OK;
    cudaError_t e = cudaSuccess;
    for (cudaStream_t s : B->side) {
        cudaError_t e1 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e1;
    }
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->origin) {
        cudaError_t e1 = cudaStreamSynchronize(B->origin);
        if (e == cudaSuccess) e = e1;
    }
    for (spect::GroupedBatch& gb : B->grouped) spect::free_grouped(gb);
    for (cudaStream_t s : B->side) cudaStreamDestroy(s);
    if (B->origin) cudaStreamDestroy(B->origin);
    for (cudaEvent_t j : B->join) cudaEventDestroy(j);
    if (B->fork) cudaEventDestroy(B->fork);
    delete B;
    if (e != cudaSuccess) return fail(SPECT_ECUDA, std::string("batch destroy: ") + cudaGetErrorString(e));
    return SPECT_OK;
}

}  // extern "C"
