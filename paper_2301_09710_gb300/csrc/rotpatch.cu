// rotpatch.cu -- rotation and attenuation of the forward projector (Section II-A,
// Algorithm 1: w = x~ * mubar) as a patch-staged kernel.
//
// One block owns an 8x8 patch of rotated-frame columns (i, j) of one view and
// walks k in runs of 16.  The bilinear corners of every sample of the patch
// lie in a small box of x_t (at most about 8*sqrt(2) + 2 on a side); the box and
// the patch's attenuation factors arrive by two 3D TMA tensor loads per k run,
// double-buffered, so the four corner reads of a sample are shared-memory
// reads instead of L2 gathers.  Weights, corner order and arithmetic are those
// of k_rot_fwd (same rotation tables), and the output is the same plane image
// W[k][C + i] with replicate halo columns: the results are bitwise the same.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <vector>

#include "spect_internal.cuh"

namespace spect {

namespace {

constexpr int kRT = 256;   // threads: 64 columns x 4 float4 groups of k
constexpr int kRP = 8;     // columns per patch side
constexpr int kRK = 16;    // k per run

// Box of x_t columns read by the samples of patch `patch` in view l: the
// clamped base corner (bi, bj) of every sample and its (+1, +1) neighbours.
__global__ void k_rot_boxes(Geometry g, int ts, const float* __restrict__ rtab, int npx, int4* boxes)
{
    __shared__ int mn_i, mn_j, mx_i, mx_j;
    const int patch = blockIdx.x, l = blockIdx.y, t = threadIdx.x;
    if (t == 0) {
        mn_i = mn_j = INT_MAX;
        mx_i = mx_j = INT_MIN;
    }
    __syncthreads();
    const int i = (patch % npx) * kRP + (t % kRP), j = (patch / npx) * kRP + (t / kRP);
    if (i < g.nx && j < g.ny) {
        const float* tab = rtab + ((size_t)l * g.ny + j) * ts;
        const int base = reinterpret_cast<const int*>(tab + 4 * g.nx)[i];
        const int bi = base % g.nx, bj = base / g.nx;
        atomicMin(&mn_i, bi);
        atomicMin(&mn_j, bj);
        atomicMax(&mx_i, bi + 1);
        atomicMax(&mx_j, bj + 1);
    }
    __syncthreads();
    if (t == 0) {
        int4 b = make_int4(0, 0, 1, 1);
        if (mx_i >= mn_i) b = make_int4(mn_i, mn_j, mx_i - mn_i + 1, mx_j - mn_j + 1);
        boxes[(size_t)patch * g.nview + l] = b;
    }
}

struct RotPatchArgs {
    Geometry g;
    int npx;             // patches along i
    int bw, bh;          // x_t box extents (the tensor map's box: 16 x bw x bh)
    int box_floats;      // bw * bh * 16
    int stage_floats;    // attenuation tile (64 * 16) + box, 128-byte multiple
    int C, wp, parea;    // plane image: halo width, row pitch, floats per plane
    int wcols;           // columns of an image row that are written (nib*16 + 2C)
    int ts;              // rotation table block per (view, row)
    int l0, nkc;         // first view of the launch; k runs
};

__global__ void __launch_bounds__(kRT) k_rot_patch(const __grid_constant__ CUtensorMap xmap,
                                                   const __grid_constant__ CUtensorMap mmap, RotPatchArgs a,
                                                   const float* __restrict__ rtab, const int4* __restrict__ boxes,
                                                   float* __restrict__ wsl, int* err)
{
    extern __shared__ __align__(128) float sm[];
    const Geometry& g = a.g;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * (size_t)a.stage_floats);
    const int patch = blockIdx.x, v = blockIdx.y, l = a.l0 + v;
    const int tid = threadIdx.x;
    const int ql = tid >> 2, k4 = tid & 3;
    const int px0 = (patch % a.npx) * kRP, py0 = (patch / a.npx) * kRP;
    const int i = px0 + (ql % kRP), j = py0 + (ql / kRP);
    const bool valid = i < g.nx && j < g.ny;
    const int4 box = boxes[(size_t)patch * g.nview + l];
    if ((smem_u32(sm) & 127u) != 0) {  // tensor copies want 128-byte aligned shared memory
        if (tid == 0 && err) atomicExch(err, (int)SPECT_ECUDA);
        return;
    }
    // stage layout: attenuation tile (8 x 8 x 16, 4 KB) then the x_t box; both 128-byte aligned
    auto issue = [&](int kc) {
        float* st = sm + (size_t)(kc & 1) * a.stage_floats;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar + (kc & 1))),
                     "r"((unsigned)(a.box_floats + kRP * kRP * kRK) * 4u)
                     : "memory");
        tma_load_3d(st, &mmap, kc * kRK, px0, l * g.ny + py0, bar + (kc & 1));
        tma_load_3d(st + kRP * kRP * kRK, &xmap, kc * kRK, box.x, box.y, bar + (kc & 1));
    };
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue(0);
        if (a.nkc > 1) issue(1);
    }
    // this column's sample: weights and the box offset of its base corner
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    int o = 0;
    if (valid) {
        const float* tab = rtab + ((size_t)l * g.ny + j) * a.ts;
        w = reinterpret_cast<const float4*>(tab)[i];
        const int base = reinterpret_cast<const int*>(tab + 4 * g.nx)[i];
        const int bi = base % g.nx, bj = base / g.nx;
        o = ((bj - box.y) * a.bw + (bi - box.x)) * kRK + 4 * k4;
    }
    const int row = a.bw * kRK;
    float* img = wsl + ((size_t)v * g.ny + j) * a.parea + a.C;
    __syncthreads();

    for (int kc = 0; kc < a.nkc; ++kc) {
        const bool ok = mbar_wait_bounded(bar + (kc & 1), (unsigned)(kc >> 1) & 1u);
        if (ok && valid) {
            const float* st = sm + (size_t)(kc & 1) * a.stage_floats;
            const float* bx = st + kRP * kRP * kRK;
            const float4 c00 = *reinterpret_cast<const float4*>(bx + o);
            const float4 c10 = *reinterpret_cast<const float4*>(bx + o + kRK);
            const float4 c01 = *reinterpret_cast<const float4*>(bx + o + row);
            const float4 c11 = *reinterpret_cast<const float4*>(bx + o + row + kRK);
            const float4 m = *reinterpret_cast<const float4*>(st + ql * kRK + 4 * k4);
            const float x00[4] = {c00.x, c00.y, c00.z, c00.w}, x10[4] = {c10.x, c10.y, c10.z, c10.w};
            const float x01[4] = {c01.x, c01.y, c01.z, c01.w}, x11[4] = {c11.x, c11.y, c11.z, c11.w};
            const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = kc * kRK + 4 * k4 + u;
                if (k >= g.nz) break;
                float va = w.x * x00[u];
                va = fmaf(w.y, x10[u], va);
                va = fmaf(w.z, x01[u], va);
                va = fmaf(w.w, x11[u], va);
                va *= mv[u];
                float* wr = img + (size_t)k * a.wp;
                wr[i] = va;
                if (i == 0)  // replicate padding along i: left halo columns
                    for (int h = -a.C; h < 0; ++h) wr[h] = va;
                if (i == g.nx - 1)  // right halo columns
                    for (int h = g.nx; h < a.wcols - a.C; ++h) wr[h] = va;
            }
        }
        if (__syncthreads_or(!ok)) {  // a copy never landed: give the ones in flight a last chance, then stop
            if (tid == 0) {
                if (err) atomicExch(err, (int)SPECT_ETIMEOUT);
                for (int u = kc; u < kc + 2 && u < a.nkc; ++u) mbar_wait_bounded(bar + (u & 1), (unsigned)(u >> 1) & 1u);
            }
            return;
        }
        if (tid == 0 && kc + 2 < a.nkc) {  // stage kc & 1 has been read by every thread
            fence_proxy_async_smem();
            issue(kc + 2);
        }
    }
}

int rot_stage_floats(int box_floats) { return (box_floats + kRP * kRP * kRK + 31) & ~31; }

size_t rot_smem(int box_floats) { return 2 * (size_t)rot_stage_floats(box_floats) * sizeof(float) + 2 * sizeof(uint64_t); }

}  // namespace

// Plan time: per-(patch, view) boxes from the rotation tables and the two
// tensor maps.  Leaves P.rotpatch = 0 when the geometry does not suit the
// kernel (k rows not a whole number of 16-byte units, boxes too large, no
// tensor-map encoder).
cudaError_t build_rotpatch(spect_plan_s& P, cudaStream_t st)
{
    P.rotpatch = 0;
    const Geometry& g = P.g;
    if (!P.fast || (g.nz % 4) != 0 || !encode_fn()) return cudaSuccess;
    // SPECT_ROTPATCH (testing): 0 = not built; 1 = built and used from the start;
    // unset = built, used once the autotuner finds it faster
    const char* env = getenv("SPECT_ROTPATCH");
    if (env && atoi(env) == 0) return cudaSuccess;
    const int npx = (g.nx + kRP - 1) / kRP, npy = (g.ny + kRP - 1) / kRP;
    const size_t nb = (size_t)npx * npy * g.nview;
    int4* boxes = nullptr;
    cudaError_t e = P.pooled ? cudaMallocAsync((void**)&boxes, nb * sizeof(int4), st)
                             : cudaMalloc((void**)&boxes, nb * sizeof(int4));
    if (e != cudaSuccess) return e;
    k_rot_boxes<<<dim3(npx * npy, g.nview), kRP * kRP, 0, st>>>(g, P.ts, P.rtab, npx, boxes);
    e = cudaGetLastError();
    std::vector<int4> hb(nb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), boxes, nb * sizeof(int4), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int bw = 1, bh = 1;
    if (e == cudaSuccess)
        for (const int4& b : hb) {
            bw = std::max(bw, b.z);
            bh = std::max(bh, b.w);
        }
    const int box_floats = bw * bh * kRK;
    CUtensorMap mx, mm;
    bool ok = e == cudaSuccess && bw <= 256 && bh <= 256 && rot_smem(box_floats) <= (size_t)P.smem_optin;
    if (ok) {
        // x_t: k (nz, contiguous) x i (nx) x j (ny)
        const cuuint64_t dx[3] = {(cuuint64_t)g.nz, (cuuint64_t)g.nx, (cuuint64_t)g.ny};
        const cuuint64_t sx[2] = {(cuuint64_t)g.nz * 4, (cuuint64_t)g.nx * g.nz * 4};
        const cuuint32_t bx[3] = {(cuuint32_t)kRK, (cuuint32_t)bw, (cuuint32_t)bh};
        // attenuation cache: k (nz) x i (nx) x (view, row) plane (nview * ny, stride ps)
        const cuuint64_t dm[3] = {(cuuint64_t)g.nz, (cuuint64_t)g.nx, (cuuint64_t)g.nview * g.ny};
        const cuuint64_t sm_[2] = {(cuuint64_t)g.nz * 4, (cuuint64_t)P.ps * 4};
        const cuuint32_t bm[3] = {(cuuint32_t)kRK, (cuuint32_t)kRP, (cuuint32_t)kRP};
        const cuuint32_t es[3] = {1, 1, 1};
        ok = encode_fn()(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, P.xt, dx, sx, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
             encode_fn()(&mm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, P.mubar, dm, sm_, bm, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if (!ok) {
        if (P.pooled) cudaFreeAsync(boxes, st);
        else cudaFree(boxes);
        return e;
    }
    P.rboxes = boxes;
    P.bytes += nb * sizeof(int4);
    P.rbw = bw;
    P.rbh = bh;
    P.rmap_x = mx;
    P.rmap_mu = mm;
    P.rotpatch = 1;
    P.rotpatch_on = env && atoi(env) == 1;
    return cudaSuccess;
}

cudaError_t launch_rot_patch(const spect_plan_s& P, int l0, int nv, cudaStream_t st)
{
    const Geometry& g = P.g;
    RotPatchArgs a;
    a.g = g;
    a.npx = (g.nx + kRP - 1) / kRP;
    a.bw = P.rbw;
    a.bh = P.rbh;
    a.box_floats = P.rbw * P.rbh * kRK;
    a.stage_floats = rot_stage_floats(a.box_floats);
    const int C = (P.bucket - 1) / 2;
    const int nib = (g.nx + 15) / 16;
    a.C = C;
    a.wp = pitch4odd(nib * 16 + 2 * C);  // as the fused kernels' untiled plane image
    a.parea = (g.nz * a.wp + 3) & ~3;
    a.wcols = nib * 16 + 2 * C;
    a.ts = P.ts;
    a.l0 = l0;
    a.nkc = (g.nz + kRK - 1) / kRK;
    const size_t smem = rot_smem(a.box_floats);
    cudaError_t e = cudaFuncSetAttribute(k_rot_patch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int npy = (g.ny + kRP - 1) / kRP;
    k_rot_patch<<<dim3(a.npx * npy, nv), kRT, smem, st>>>(P.rmap_x, P.rmap_mu, a, P.rtab, P.rboxes, P.slab, P.err);
    return cudaGetLastError();
}

}  // namespace spect
