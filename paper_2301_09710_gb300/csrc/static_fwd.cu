// static_fwd.cu -- spect_forward_static: the forward projection v = A x for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: real-time or embedded hosts
// whose device memory is reserved up front and may not grow while they run,
// and plug-in environments (a host application's image pipeline, say) that
// hand out device buffers but own the allocator, so a library must not take
// memory behind their back.  For them this entry point runs the low-memory separable-PSF
// kernels (rotate + attenuate into a work slab, then blur + depth sum) with
// the slab and the per-view rotation constants in file-scope __device__
// arrays of fixed size, instead of a plan.  The caller passes every input and
// the output; nothing is allocated, neither here nor in a library it calls.
//
// Limits: nx*ny*nz <= kScratchFloats (8 Mi voxels, 32 MiB of slab) and
// nview <= kScratchViews.  The arrays live on every device that loads the
// library until the process exits.  All calls share them, so calls that
// overlap on the GPU (other streams, other host threads) race: serialise
// them.  Nothing needs to start at zero: each call writes every slab element
// and every rotation constant it reads.
#include <mutex>

#include "spect_internal.cuh"

namespace {

constexpr size_t kScratchFloats = (size_t)8 << 20;  // 8 Mi floats = 32 MiB
constexpr int kScratchViews = 4096;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_scratch_slab[kScratchFloats];
static __device__ __align__(256) spect::ViewRot g_scratch_rot[kScratchViews];

std::mutex g_lock;
float* g_slab_addr[kMaxDevices];           // device address of g_scratch_slab, per device
spect::ViewRot* g_rot_addr[kMaxDevices];   // device address of g_scratch_rot, per device
spect::ViewRot g_rot_host[kScratchViews];  // host staging of the constants (guarded by g_lock)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Device addresses of the scratch arrays on `dev` (the current device),
// looked up once per device.  In host code the array names are host-side
// stand-ins, not device addresses.
spect_status scratch_addresses(int dev, float** slab, spect::ViewRot** rot)
{
    if (dev < 0 || dev >= kMaxDevices) return spect::set_error(SPECT_EUNSUPPORTED, "device ordinal out of range");
    if (!g_slab_addr[dev]) {
        void* a = nullptr;
        void* b = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, g_scratch_slab);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&b, g_scratch_rot);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return spect::set_error(SPECT_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        g_slab_addr[dev] = static_cast<float*>(a);
        g_rot_addr[dev] = static_cast<spect::ViewRot*>(b);
    }
    *slab = g_slab_addr[dev];
    *rot = g_rot_addr[dev];
    return SPECT_OK;
}

}  // namespace

extern "C" spect_status spect_forward_static(int nx, int ny, int nz, int nview, const float* x, const float* mu,
                                             float dy, const float* psf_fx, const float* psf_fz, int px, int pz,
                                             int nview_psf, const double* angles, float* v, spect_stream stream)
{
    using spect::set_error;
    if (nx != ny) return set_error(SPECT_EINVAL, "nx must equal ny (rotation in the x-y plane)");
    if (nx < 2 || nx > 1024) return set_error(SPECT_EINVAL, "nx must be in [2, 1024]");
    if (nz < 1 || nz > 4096) return set_error(SPECT_EINVAL, "nz must be in [1, 4096]");
    if (nview < 1 || nview > kScratchViews) return set_error(SPECT_EINVAL, "nview must be in [1, 4096]");
    if (px < 1 || pz < 1 || px > 127 || pz > 127 || (px % 2) == 0 || (pz % 2) == 0)
        return set_error(SPECT_EINVAL, "PSF sizes px, pz must be odd and in [1, 127]");
    if (nview_psf != 1 && nview_psf != nview) return set_error(SPECT_EINVAL, "nview_psf must be 1 or nview");
    if (!(dy >= 0.f) || !isfinite(dy)) return set_error(SPECT_EINVAL, "dy must be finite and >= 0");
    if (!x || !v || !psf_fx || !psf_fz) return set_error(SPECT_EINVAL, "x, v, psf_fx and psf_fz must not be NULL");
    const void* ptrs[] = {x, v, psf_fx, psf_fz, mu};
    for (const void* p : ptrs)
        if (p && !aligned16(p)) return set_error(SPECT_EINVAL, "device buffers must be 16-byte aligned");
    const size_t vol = (size_t)nx * ny * nz;
    if (vol > kScratchFloats)
        return set_error(SPECT_EINVAL, "nx*ny*nz exceeds the static scratch of spect_forward_static (8388608 voxels)");
    if (angles)
        for (int l = 0; l < nview; ++l)
            if (!isfinite(angles[l])) return set_error(SPECT_EINVAL, "angles must be finite");

    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return set_error(SPECT_ECUDA, "device query failed");
    }

    // A plan description on the host stack pointing at the caller's buffers and
    // the static scratch (its containers stay empty: no allocation).
    spect_plan_s P;
    spect::Geometry& g = P.g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.nview = nview;
    g.px = px; g.pz = pz; g.nvp = nview_psf;
    g.cint = (nx - 1) / 2;
    g.cfrac = (nx - 1) % 2 ? 0.5f : 0.f;
    g.dy = dy;
    g.has_mu = mu != nullptr;
    P.separable = 1;
    P.cls_z = nz >= 2 ? 3 : 1;
    P.sep_tk = spect::choose_sep_tile(g, P.cls_z, (size_t)smem_optin);
    if (P.sep_tk < 1) return set_error(SPECT_EUNSUPPORTED, "separable PSF tile does not fit shared memory");
    P.mu = const_cast<float*>(mu);
    P.fx = const_cast<float*>(psf_fx);
    P.fz = const_cast<float*>(psf_fz);
    P.chunk = (int)std::min<size_t>((size_t)nview, kScratchFloats / vol);

    std::lock_guard<std::mutex> lk(g_lock);
    spect_status r = scratch_addresses(dev, &P.slab, &P.rot);
    if (r != SPECT_OK) return r;
    spect::make_view_rot(nx, nview, angles, g_rot_host);
    // pageable source: the copy is staged before the call returns, so the host
    // array may be rewritten by the next call
    cudaError_t e = cudaMemcpyAsync(P.rot, g_rot_host, sizeof(spect::ViewRot) * nview, cudaMemcpyHostToDevice, st);
    for (int l0 = 0; e == cudaSuccess && l0 < nview; l0 += P.chunk) {
        const int nv = std::min(P.chunk, nview - l0);
        e = spect::launch_rotate_atten(P, x, l0, nv, st);
        if (e == cudaSuccess) e = spect::launch_conv_forward(P, v, l0, nv, nullptr, nullptr, st);
    }
    if (e != cudaSuccess) return set_error(SPECT_ECUDA, cudaGetErrorString(e));
    return SPECT_OK;
}
