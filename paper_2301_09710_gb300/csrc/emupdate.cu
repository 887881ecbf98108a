// emupdate.cu -- the element-wise parts of one EM iteration (Eqs. (7)-(8) of
// arXiv 2301.09710) as stand-alone kernels with their gradients, for training
// through an unrolled reconstruction (Algorithm 3): the projector parts A and A'
// are the plan's kernels, these are the steps between them.
//
//   ratio    r = y / (ybar + rbar), 0 where ybar + rbar <= 0 (the guard of the
//            fused EM step);
//   update   x+ = the non-negative root of beta x+^2 + d x+ - x e = 0,
//            d = s - beta u (beta = 0: x e / s), the em_update() of the fused
//            kernels, bit for bit.
//
// Gradients (vector-Jacobian products).  Ratio: dr/dybar = -r / (ybar + rbar).
// Update: differentiating beta x+^2 + d x+ - x e = 0 implicitly,
//   (2 beta x+ + d) dx+ = e dx + x de + beta x+ du,
// and 2 beta x+ + d = sqrt(d^2 + 4 beta x e) =: q (q = s at beta = 0), so
//   dx+/dx = e / q,  dx+/de = x / q,  dx+/du = beta x+ / q,
// and zero wherever the forward guard set x+ to 0.  Element-wise and HBM-bound:
// float4 accesses for the ratio when n and the pointers allow; grid-stride loops
// over at most 8 blocks per SM.
#include <algorithm>
#include <cmath>

#include "spect_internal.cuh"

namespace spect {
namespace {

constexpr int kEwThreads = 256;

__device__ __forceinline__ float ratio_of(float yb_proj, float y, float rb)
{
    const float yb = yb_proj + rb;
    return yb > 0.f ? y / yb : 0.f;
}

// dL/dybar for one element, given dL/dratio
__device__ __forceinline__ float ratio_vjp(float yb_proj, float y, float rb, float g)
{
    const float yb = yb_proj + rb;
    if (!(yb > 0.f)) return 0.f;
    const float r = y / yb;
    return -g * r / yb;
}

// the update's partial derivatives (e / q, x / q, beta x+ / q), zero where the
// forward guard applies (same branches as em_update)
__device__ __forceinline__ void update_vjp(float x, float e, float s, float u, float beta, float g, float& gx,
                                           float& ge, float& gu)
{
    gx = ge = gu = 0.f;
    if (beta == 0.f) {
        if (s > 0.f) {
            gx = g * e / s;
            ge = g * x / s;
        }
        return;
    }
    const float xe = x * e;
    const float d = fmaf(-beta, u, s);  // as em_update
    const float q = sqrtf(fmaf(d, d, 4.f * beta * xe));
    if (d >= 0.f && !(d + q > 0.f)) return;  // x+ set to 0 by the guard
    if (!(q > 0.f)) return;
    const float xp = em_update(x, e, s, u, beta);
    gx = g * e / q;
    ge = g * x / q;
    gu = g * beta * xp / q;
}

__global__ void __launch_bounds__(kEwThreads) k_em_ratio(size_t n, const float* __restrict__ ybar,
                                                        const float* __restrict__ y, const float* __restrict__ rbar,
                                                        const float* __restrict__ g, float* __restrict__ out)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float rb = rbar ? rbar[i] : 0.f;
        out[i] = g ? ratio_vjp(ybar[i], y[i], rb, g[i]) : ratio_of(ybar[i], y[i], rb);
    }
}

__global__ void __launch_bounds__(kEwThreads) k_em_ratio4(size_t n4, const float4* __restrict__ ybar,
                                                         const float4* __restrict__ y,
                                                         const float4* __restrict__ rbar,
                                                         const float4* __restrict__ g, float4* __restrict__ out)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 a = ybar[i], b = y[i];
        const float4 r = rbar ? rbar[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 o;
        if (g) {
            const float4 gg = g[i];
            o = make_float4(ratio_vjp(a.x, b.x, r.x, gg.x), ratio_vjp(a.y, b.y, r.y, gg.y),
                            ratio_vjp(a.z, b.z, r.z, gg.z), ratio_vjp(a.w, b.w, r.w, gg.w));
        } else {
            o = make_float4(ratio_of(a.x, b.x, r.x), ratio_of(a.y, b.y, r.y), ratio_of(a.z, b.z, r.z),
                            ratio_of(a.w, b.w, r.w));
        }
        out[i] = o;
    }
}

__global__ void __launch_bounds__(kEwThreads) k_em_update(size_t n, const float* __restrict__ x,
                                                         const float* __restrict__ e, const float* __restrict__ s,
                                                         const float* __restrict__ u, float beta,
                                                         float* __restrict__ out)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = em_update(x[i], e[i], s[i], u ? u[i] : 0.f, beta);
}

__global__ void __launch_bounds__(kEwThreads) k_em_update_vjp(size_t n, const float* __restrict__ x,
                                                             const float* __restrict__ e,
                                                             const float* __restrict__ s,
                                                             const float* __restrict__ u, float beta,
                                                             const float* __restrict__ g, float* __restrict__ gx,
                                                             float* __restrict__ ge, float* __restrict__ gu)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float a, b, c;
        update_vjp(x[i], e[i], s[i], u ? u[i] : 0.f, beta, g[i], a, b, c);
        if (gx) gx[i] = a;
        if (ge) ge[i] = b;
        if (gu) gu[i] = c;
    }
}

unsigned ew_blocks(size_t n)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t want = (n + kEwThreads - 1) / kEwThreads;
    const size_t cap = (size_t)std::max(sms, 1) * 8;
    return (unsigned)std::max<size_t>(1, std::min(want, cap));
}

bool a16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

spect_status launched(const char* what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(SPECT_ECUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
    return SPECT_OK;
}

}  // namespace
}  // namespace spect

extern "C" {

spect_status spect_em_ratio(size_t n, const float* ybar, const float* y, const float* rbar, float* ratio,
                            spect_stream stream)
{
    using namespace spect;
    if (n == 0) return SPECT_OK;
    if (!ybar || !y || !ratio) return set_error(SPECT_EINVAL, "ybar, y and ratio must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (n % 4 == 0 && a16(ybar) && a16(y) && a16(ratio) && (!rbar || a16(rbar)))
        k_em_ratio4<<<ew_blocks(n / 4), kEwThreads, 0, st>>>(
            n / 4, reinterpret_cast<const float4*>(ybar), reinterpret_cast<const float4*>(y),
            reinterpret_cast<const float4*>(rbar), nullptr, reinterpret_cast<float4*>(ratio));
    else
        k_em_ratio<<<ew_blocks(n), kEwThreads, 0, st>>>(n, ybar, y, rbar, nullptr, ratio);
    return launched("EM ratio launch");
}

spect_status spect_em_ratio_backward(size_t n, const float* ybar, const float* y, const float* rbar,
                                     const float* g_ratio, float* g_ybar, spect_stream stream)
{
    using namespace spect;
    if (n == 0) return SPECT_OK;
    if (!ybar || !y || !g_ratio || !g_ybar)
        return set_error(SPECT_EINVAL, "ybar, y, g_ratio and g_ybar must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (n % 4 == 0 && a16(ybar) && a16(y) && a16(g_ratio) && a16(g_ybar) && (!rbar || a16(rbar)))
        k_em_ratio4<<<ew_blocks(n / 4), kEwThreads, 0, st>>>(
            n / 4, reinterpret_cast<const float4*>(ybar), reinterpret_cast<const float4*>(y),
            reinterpret_cast<const float4*>(rbar), reinterpret_cast<const float4*>(g_ratio),
            reinterpret_cast<float4*>(g_ybar));
    else
        k_em_ratio<<<ew_blocks(n), kEwThreads, 0, st>>>(n, ybar, y, rbar, g_ratio, g_ybar);
    return launched("EM ratio gradient launch");
}

spect_status spect_em_update(size_t n, const float* x, const float* e, const float* s, const float* u, float beta,
                             float* out, spect_stream stream)
{
    using namespace spect;
    if (n == 0) return SPECT_OK;
    if (!x || !e || !s || !out) return set_error(SPECT_EINVAL, "x, e, s and out must not be NULL");
    if (!(beta >= 0.f) || !isfinite(beta)) return set_error(SPECT_EINVAL, "beta must be finite and >= 0");
    if (beta > 0.f && !u) return set_error(SPECT_EINVAL, "u is required when beta > 0");
    k_em_update<<<ew_blocks(n), kEwThreads, 0, (cudaStream_t)stream>>>(n, x, e, s, beta > 0.f ? u : nullptr, beta,
                                                                       out);
    return launched("EM update launch");
}

spect_status spect_em_update_backward(size_t n, const float* x, const float* e, const float* s, const float* u,
                                      float beta, const float* g_out, float* g_x, float* g_e, float* g_u,
                                      spect_stream stream)
{
    using namespace spect;
    if (n == 0) return SPECT_OK;
    if (!x || !e || !s || !g_out) return set_error(SPECT_EINVAL, "x, e, s and g_out must not be NULL");
    if (!(beta >= 0.f) || !isfinite(beta)) return set_error(SPECT_EINVAL, "beta must be finite and >= 0");
    if (beta > 0.f && !u) return set_error(SPECT_EINVAL, "u is required when beta > 0");
    k_em_update_vjp<<<ew_blocks(n), kEwThreads, 0, (cudaStream_t)stream>>>(
        n, x, e, s, beta > 0.f ? u : nullptr, beta, g_out, g_x, g_e, beta > 0.f ? g_u : nullptr);
    if (beta == 0.f && g_u) cudaMemsetAsync(g_u, 0, n * sizeof(float), (cudaStream_t)stream);
    return launched("EM update gradient launch");
}

}  // extern "C"
