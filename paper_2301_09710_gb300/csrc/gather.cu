// gather.cu -- adjoint rotation and view sum of A' (Section II-A, Algorithm 2)
// as a patch-staged gather:
//
//   x_t(q, k) = sum_l sum_{(p, w) in adj(l, q)} w * t_l(p, k)
//
// One block owns an 8x8 patch of destination columns q and a run of KC
// consecutive k.  For every view, the source pixels its destinations read lie
// in a small box of the rotated frame (at most about 8*sqrt(2) + 2 on a side);
// the box is brought into shared memory by one TMA tensor load (3D tile of the
// t slab: k x i x plane) and the patch's adjacency entries by one bulk copy,
// several views ahead of use, so the gathers read shared memory instead of
// waiting on L2.  The entries hold box-local offsets computed at plan time from
// the fixed-length lists k_build_adjacency_fixed writes (same weights, same
// order), and the per-view sum and the Kahan sum over views are those of
// k_adj_rot_t: the results are bitwise the same.
#include <cuda.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <vector>

#include "spect_internal.cuh"

namespace spect {

namespace {

constexpr int kGT = 256;      // threads: 64 destinations x 4 float4 groups of k
constexpr int kPatch = 8;     // destinations per patch side
constexpr int kStages = 3;    // views in flight per block (measured best: 3 of 3, 4, 6, 8)

// Box of source pixels read by patch `patch` in view l: (i0, j0, width, height).
__global__ void k_patch_boxes(Geometry g, int ps, int maxe, const AdjEntry* __restrict__ adjf, int npx, int4* boxes)
{
    __shared__ int mn_i, mn_j, mx_i, mx_j;
    const int patch = blockIdx.x, l = blockIdx.y, t = threadIdx.x;
    if (t == 0) {
        mn_i = mn_j = INT_MAX;
        mx_i = mx_j = INT_MIN;
    }
    __syncthreads();
    const int qi = (patch % npx) * kPatch + (t % kPatch), qj = (patch / npx) * kPatch + (t / kPatch);
    if (qi < g.nx && qj < g.ny) {
        const AdjEntry* e = adjf + ((size_t)(qj * g.nx + qi) * g.nview + l) * maxe;
        for (int m = 0; m < maxe; ++m) {
            if (e[m].w == 0.f) continue;
            const int pj = e[m].p / ps, pi = (e[m].p - pj * ps) / g.nz;
            atomicMin(&mn_i, pi);
            atomicMin(&mn_j, pj);
            atomicMax(&mx_i, pi);
            atomicMax(&mx_j, pj);
        }
    }
    __syncthreads();
    if (t == 0) {
        int4 b = make_int4(0, 0, 0, 0);
        if (mx_i >= mn_i) b = make_int4(mn_i, mn_j, mx_i - mn_i + 1, mx_j - mn_j + 1);
        boxes[(size_t)patch * g.nview + l] = b;
    }
}

// Patch entries [patch][l][64][maxe]: (box-local offset (row*BW + col)*KC, weight);
// zero entries for padding and for destinations outside the image.
__global__ void k_patch_entries(Geometry g, int ps, int maxe, const AdjEntry* __restrict__ adjf, int npx,
                                const int4* __restrict__ boxes, int bw, int kc, AdjEntry* pent)
{
    const int patch = blockIdx.x, l = blockIdx.y, t = threadIdx.x;
    const int qi = (patch % npx) * kPatch + (t % kPatch), qj = (patch / npx) * kPatch + (t / kPatch);
    const int4 b = boxes[(size_t)patch * g.nview + l];
    AdjEntry* out = pent + (((size_t)patch * g.nview + l) * (kPatch * kPatch) + t) * maxe;
    const bool inside = qi < g.nx && qj < g.ny;
    const AdjEntry* e = adjf + ((size_t)(qj * g.nx + qi) * g.nview + l) * maxe;
    for (int m = 0; m < maxe; ++m) {
        AdjEntry o;  // padding and outside destinations: weight 0 on the box's first element
        o.p = 0;
        o.w = 0.f;
        if (inside && e[m].w != 0.f) {
            const int pj = e[m].p / ps, pi = (e[m].p - pj * ps) / g.nz;
            o.p = ((pj - b.y) * bw + (pi - b.x)) * kc;
            o.w = e[m].w;
        }
        out[m] = o;
    }
}

struct GatherArgs {
    Geometry g;
    int npx;         // patches along i
    int bw, bh, kc;  // box extents (the tensor map's box: kc x bw x bh)
    int box_floats;  // bw * bh * kc
    int ent_bytes;   // 64 * maxe * 8
    int stage_floats;
    int l0, nv;      // views [l0, l0 + nv) of the plan; slab view v holds view l0 + v
    int nkc;         // runs of kc depth rows per patch
};

// Consumer threads: 64 destinations x 4 float4 groups of k; one more warp
// produces: it refills a stage as soon as every consumer has released it
// (per-stage "empty" barrier), so consumers never meet at a block barrier
// inside the view loop.
template <int MAXE>
__device__ __forceinline__ void adj_gather_body(const CUtensorMap* tmap, const GatherArgs& a,
                                                const int4* __restrict__ boxes, const AdjEntry* __restrict__ pent,
                                                float* out, int accumulate, const EmArgs& em, int* err,
                                                const int patch, const int kcb)
{
    extern __shared__ __align__(128) float sm[];
    const Geometry& g = a.g;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)kStages * a.stage_floats);
    uint64_t* empty = full + kStages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kStages);
    const int kc0 = kcb * a.kc;
    const int tid = threadIdx.x;
    const bool producer = tid >= kGT;

    // tensor copies want 128-byte aligned shared memory: refuse (error word) rather than fault
    if ((smem_u32(sm) & 127u) != 0) {
        if (tid == 0 && err) atomicExch(err, (int)SPECT_ECUDA);
        return;
    }
    if (tid == kGT) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, kGT);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (producer) {
        if (tid != kGT) return;  // one lane issues
        int issued = 0;
        for (int v = 0; v < a.nv; ++v) {
            const int s = v % kStages;
            if (*abort_flag) break;
            if (v >= kStages && !mbar_wait_bounded(empty + s, (unsigned)(v / kStages - 1) & 1u)) {
                *abort_flag = 1;
                break;
            }
            if (v >= kStages) fence_proxy_async_smem();
            float* st = sm + (size_t)s * a.stage_floats;
            const int l = a.l0 + v;
            const int4 b = boxes[(size_t)patch * g.nview + l];
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(full + s)),
                         "r"((unsigned)(a.box_floats * 4 + a.ent_bytes))
                         : "memory");
            tma_load_3d(st, tmap, kc0, b.x, v * g.ny + b.y, full + s);
            tma_copy_1d(st + a.box_floats, pent + ((size_t)patch * g.nview + l) * (kPatch * kPatch) * MAXE,
                        (unsigned)a.ent_bytes, full + s);
            issued = v + 1;
        }
        if (*abort_flag) {  // let every copy in flight land before the block's shared memory is released
            if (err) atomicExch(err, (int)SPECT_ETIMEOUT);
            for (int u = issued - kStages < 0 ? 0 : issued - kStages; u < issued; ++u)
                mbar_wait_bounded(full + (u % kStages), (unsigned)(u / kStages) & 1u);
        }
        return;
    }

    const int ql = tid >> 2, k4 = tid & 3;  // destination in the patch, float4 group of k
    const int qi = (patch % a.npx) * kPatch + (ql % kPatch), qj = (patch / a.npx) * kPatch + (ql / kPatch);
    // the EM epilogue's operands, fetched before the view loop so their latency hides behind it
    const int k = kc0 + 4 * k4;
    const bool mine = qi < g.nx && qj < g.ny && k < g.nz;
    const size_t o = mine ? (size_t)(qj * g.nx + qi) * g.nz + k : 0;
    float4 ex = make_float4(0.f, 0.f, 0.f, 0.f), es = ex, eu = ex;
    if (mine && em.x) {
        ex = *reinterpret_cast<const float4*>(em.x + o);
        es = *reinterpret_cast<const float4*>(em.s + o);
        if (em.u) eu = *reinterpret_cast<const float4*>(em.u + o);
    }

    KSum acc[4];
    bool failed = false;
    for (int v = 0; v < a.nv; ++v) {
        const int s = v % kStages;
        if (!failed) {
            if (mbar_wait_bounded(full + s, (unsigned)(v / kStages) & 1u)) {
                const float* box = sm + (size_t)s * a.stage_floats;
                const AdjEntry* e = reinterpret_cast<const AdjEntry*>(box + a.box_floats) + ql * MAXE;
                AdjEntry en[MAXE];
#pragma unroll
                for (int m = 0; m < MAXE; ++m) en[m] = e[m];
                float4 tv[MAXE];
#pragma unroll
                for (int m = 0; m < MAXE; ++m) tv[m] = *reinterpret_cast<const float4*>(box + en[m].p + 4 * k4);
                float sv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int m = 0; m < MAXE; ++m) {
                    sv[0] = fmaf(en[m].w, tv[m].x, sv[0]);
                    sv[1] = fmaf(en[m].w, tv[m].y, sv[1]);
                    sv[2] = fmaf(en[m].w, tv[m].z, sv[2]);
                    sv[3] = fmaf(en[m].w, tv[m].w, sv[3]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u].add(sv[u]);
            } else {
                failed = true;
                *abort_flag = 1;
            }
        }
        // release the stage (also after a failed wait, so the producer never waits on it)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(empty + s)) : "memory");
    }
    if (failed || *abort_flag) return;

    if (!mine) return;
    const float xv[4] = {ex.x, ex.y, ex.z, ex.w}, sv4[4] = {es.x, es.y, es.z, es.w}, uv[4] = {eu.x, eu.y, eu.z, eu.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        float val = acc[u].value();
        if (accumulate) val += out[o + u];
        if (em.x) em.x[o + u] = em_update(xv[u], val, sv4[u], uv[u], em.beta);
        else out[o + u] = val;
    }
}

template <int MAXE>
__global__ void __launch_bounds__(kGT + 32) k_adj_gather(const __grid_constant__ CUtensorMap tmap, GatherArgs a,
                                                         const int4* __restrict__ boxes,
                                                         const AdjEntry* __restrict__ pent, float* out,
                                                         int accumulate, EmArgs em, int* err)
{
    // the k runs of a patch are adjacent blocks, so they run side by side and the
    // patch's entries, which each of them reads, come from DRAM about once
    // (0.246 -> 0.213 ms per 128-view launch against the patch-major order)
    const int patch = (int)blockIdx.x / a.nkc, kcb = (int)blockIdx.x - patch * a.nkc;
    adj_gather_body<MAXE>(&tmap, a, boxes, pent, out, accumulate, em, err, patch, kcb);
}


// floats per pipeline stage: the box, then the entries, rounded up to 128 bytes
int stage_floats(int box_floats, int ent_bytes) { return (box_floats + ent_bytes / 4 + 31) & ~31; }

size_t gather_smem(int box_floats, int ent_bytes)
{
    // stages | full and empty barriers | abort flag
    return (size_t)kStages * stage_floats(box_floats, ent_bytes) * sizeof(float) + 2 * kStages * sizeof(uint64_t) +
           16;
}

// One plan's arguments of the grouped gather (the tensor map in the kernel's
// parameter space, as in the per-plan launch).
struct GroupGather {
    CUtensorMap tmap;
    GatherArgs a;
    const int4* boxes;
    const AdjEntry* pent;
    float* out;
    EmArgs em;
    int accumulate;
    int* err;
};
struct GroupGathers {
    GroupGather p[kGroupMax];
    GroupGrid grid;
};

template <int MAXE>
__global__ void __launch_bounds__(kGT + 32) k_adj_gather_grp(const __grid_constant__ GroupGathers gg)
{
    const int4 w = group_item(gg.grid);
    const GroupGather& q = gg.p[w.x];
    adj_gather_body<MAXE>(&q.tmap, q.a, q.boxes, q.pent, q.out, q.accumulate, q.em, q.err, w.z, w.y);
}

}  // namespace

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        cudaGetLastError();
    }
    return fn;
}

int gather_kc() { return 16; }

// Plan time: boxes, box extents and patch entries.  Leaves P.gather = 0 when
// the geometry does not suit the kernel (k rows not a whole number of 16-byte
// units, boxes too large for the tensor map or shared memory, no encoder).
cudaError_t build_gather(spect_plan_s& P, cudaStream_t st)
{
    P.gather = 0;
    const Geometry& g = P.g;
    if (!P.fast || (g.nz % 4) != 0 || !encode_fn()) return cudaSuccess;
    const char* env = getenv("SPECT_GATHER");  // 0: use the list gather k_adj_rot_t (testing)
    if (env && atoi(env) == 0) return cudaSuccess;
    const int npx = (g.nx + kPatch - 1) / kPatch, npy = (g.ny + kPatch - 1) / kPatch;
    const size_t nb = (size_t)npx * npy * g.nview;
    int4* boxes = nullptr;
    cudaError_t e = P.pooled ? cudaMallocAsync((void**)&boxes, nb * sizeof(int4), st)
                             : cudaMalloc((void**)&boxes, nb * sizeof(int4));
    if (e != cudaSuccess) return e;
    k_patch_boxes<<<dim3(npx * npy, g.nview), kPatch * kPatch, 0, st>>>(g, P.ps, P.adj_max, P.adjf, npx, boxes);
    e = cudaGetLastError();
    std::vector<int4> hb(nb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), boxes, nb * sizeof(int4), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        if (P.pooled) cudaFreeAsync(boxes, st);
        else cudaFree(boxes);
        return e;
    }
    int bw = 1, bh = 1;
    for (const int4& b : hb) {
        bw = std::max(bw, b.z);
        bh = std::max(bh, b.w);
    }
    const int kc = gather_kc();
    const int box_floats = bw * bh * kc;
    const int ent_bytes = kPatch * kPatch * P.adj_max * (int)sizeof(AdjEntry);
    if (bw > 256 || bh > 256 || gather_smem(box_floats, ent_bytes) > (size_t)P.smem_optin ||
        (size_t)box_floats * 4 + ent_bytes >= (1u << 20)) {
        if (P.pooled) cudaFreeAsync(boxes, st);
        else cudaFree(boxes);
        return cudaSuccess;
    }
    const size_t nent = nb * kPatch * kPatch * P.adj_max;
    AdjEntry* pent = nullptr;
    e = P.pooled ? cudaMallocAsync((void**)&pent, nent * sizeof(AdjEntry), st)
                 : cudaMalloc((void**)&pent, nent * sizeof(AdjEntry));
    if (e != cudaSuccess) {
        if (P.pooled) cudaFreeAsync(boxes, st);
        else cudaFree(boxes);
        return e;
    }
    k_patch_entries<<<dim3(npx * npy, g.nview), kPatch * kPatch, 0, st>>>(g, P.ps, P.adj_max, P.adjf, npx, boxes,
                                                                         bw, kc, pent);
    e = cudaGetLastError();
    P.gboxes = boxes;
    P.gent = pent;
    P.bytes += nb * sizeof(int4) + nent * sizeof(AdjEntry);
    P.gbw = bw;
    P.gbh = bh;
    P.gnpx = npx;
    P.gnpy = npy;
    P.gather = e == cudaSuccess;
    return e;
}

namespace {
// The t slab as a 3D tensor map -- k (nz, contiguous) x i (nx, stride nz) x
// plane (chunk * ny, stride ps) -- and the gather's arguments for views
// [l0, l0 + nv).
cudaError_t gather_setup(const spect_plan_s& P, int l0, int nv, CUtensorMap* map, GatherArgs* a)
{
    const Geometry& g = P.g;
    const int kc = gather_kc();
    const cuuint64_t dims[3] = {(cuuint64_t)g.nz, (cuuint64_t)g.nx, (cuuint64_t)P.chunk * g.ny};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nz * 4, (cuuint64_t)P.ps * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kc, (cuuint32_t)P.gbw, (cuuint32_t)P.gbh};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, P.slab, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    a->g = g;
    a->npx = P.gnpx;
    a->bw = P.gbw;
    a->bh = P.gbh;
    a->kc = kc;
    a->box_floats = P.gbw * P.gbh * kc;
    a->ent_bytes = kPatch * kPatch * P.adj_max * (int)sizeof(AdjEntry);
    a->stage_floats = stage_floats(a->box_floats, a->ent_bytes);
    a->l0 = l0;
    a->nv = nv;
    a->nkc = (g.nz + kc - 1) / kc;
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_adj_gather(const spect_plan_s& P, int l0, int nv, float* out, int accumulate, EmArgs em,
                              cudaStream_t st)
{
    CUtensorMap map;
    GatherArgs a;
    cudaError_t es = gather_setup(P, l0, nv, &map, &a);
    if (es != cudaSuccess) return es;
    const size_t smem = gather_smem(a.box_floats, a.ent_bytes);
    const dim3 grid(P.gnpx * P.gnpy * a.nkc);  // (patch, k run), the k runs of a patch adjacent
    switch (P.adj_max) {
#define SPECT_G(M)                                                                                           \
    case M: {                                                                                                \
        cudaError_t e = cudaFuncSetAttribute(k_adj_gather<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                             (int)smem);                                                     \
        if (e != cudaSuccess) return e;                                                                      \
        k_adj_gather<M><<<grid, kGT + 32, smem, st>>>(map, a, P.gboxes, P.gent, out, accumulate, em, P.err); \
        break;                                                                                               \
    }
        SPECT_G(1) SPECT_G(2) SPECT_G(3) SPECT_G(4) SPECT_G(5) SPECT_G(6) SPECT_G(7) SPECT_G(8)
#undef SPECT_G
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The grouped gather of a batch: per adjacency-list length, one launch over
// every plan's (patch, k run) blocks, largest plans first; each plan's MLEM
// update (beta = 0) in the epilogue, as in its own EM step.
cudaError_t build_grouped_gather(const std::vector<spect_plan_s*>& plans, GroupedBatch& B,
                                 std::vector<GroupLaunch>& out)
{
    (void)B;
    for (int maxe = 1; maxe <= 8; ++maxe) {
        std::vector<int> idx;
        for (int i = 0; i < (int)plans.size(); ++i)
            if (plans[i]->adj_max == maxe) idx.push_back(i);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
            const auto w = [](const spect_plan_s* P) { return (size_t)P->g.nx * P->g.ny * P->g.nz * P->g.nview; };
            return w(plans[x]) > w(plans[y]);
        });
        for (size_t c0 = 0; c0 < idx.size(); c0 += kGroupMax) {
            const size_t c1 = std::min(idx.size(), c0 + (size_t)kGroupMax);
            GroupGathers gg{};
            size_t smem = 0;
            for (size_t m = c0; m < c1; ++m) {
                const spect_plan_s& P = *plans[idx[m]];
                GroupGather& q = gg.p[m - c0];
                cudaError_t e = gather_setup(P, 0, P.g.nview, &q.tmap, &q.a);
                if (e != cudaSuccess) return e;
                q.boxes = P.gboxes;
                q.pent = P.gent;
                q.out = P.et;
                q.em.x = P.xt;
                q.em.s = P.st;
                q.em.u = nullptr;
                q.em.beta = 0.f;
                q.accumulate = 0;
                q.err = P.err;
                smem = std::max(smem, gather_smem(q.a.box_floats, q.a.ent_bytes));
                // the gather's grid: (run of kc depth rows, patch), the k runs of a patch adjacent
                const int mm = (int)(m - c0), nkc = q.a.nkc;
                if (mm == 0) gg.grid.first[0] = 0;
                gg.grid.gx[mm] = nkc;
                gg.grid.gy[mm] = P.gnpx * P.gnpy;
                gg.grid.first[mm + 1] = gg.grid.first[mm] + P.gnpx * P.gnpy * nkc;
                gg.grid.n = mm + 1;
            }
            const unsigned nb = (unsigned)gg.grid.first[gg.grid.n];
            GroupLaunch L;
            switch (maxe) {
#define SPECT_GG(M)                                                                                            \
    case M:                                                                                                    \
        L = [gg, nb, smem](cudaStream_t st) -> cudaError_t {                                                   \
            cudaError_t e2 = cudaFuncSetAttribute(k_adj_gather_grp<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                  (int)smem);                                                  \
            if (e2 != cudaSuccess) return e2;                                                                  \
            k_adj_gather_grp<M><<<nb, kGT + 32, smem, st>>>(gg);                                                \
            return cudaGetLastError();                                                                         \
        };                                                                                                     \
        break;
                SPECT_GG(1) SPECT_GG(2) SPECT_GG(3) SPECT_GG(4) SPECT_GG(5) SPECT_GG(6) SPECT_GG(7) SPECT_GG(8)
#undef SPECT_GG
                default: return cudaErrorInvalidValue;
            }
            out.push_back(L);
        }
    }
    return cudaSuccess;
}

}  // namespace spect
