// grouped.cu -- EM iterations of many plans as grouped launches (the batch
// interface spect_batch_*): one launch per stage and kernel variant over a work
// list that spans every plan of the batch, instead of one launch per stage and
// plan.  Stages of one EM iteration (Eqs. (7)-(8), beta = 0):
//   rotation + attenuation (per PSF bucket, attenuation staged or not),
//   blur + depth-group sums (per bucket, tiled or not), depth-group reduce with
//   the EM ratio (all plans), blur adjoint + attenuation (per bucket, tiled or
//   not), adjoint rotation + view sum + MLEM update (gather.cu, per list length),
// plus the layout transposes of the iterates before the first and after the
// last iteration.  A block finds its plan and its coordinates in that plan's own
// grid from blockIdx.x (the plans' block ranges are in the launch parameters);
// the plan's arguments come from a __grid_constant__ parameter array, and the block runs
// the same device body as the plan's own launch (fused_body.cuh), so every plan
// gets bitwise the values it gets alone.  The largest plans' blocks come first,
// so their long blocks start early and small plans fill the tail.
#include <algorithm>
#include <numeric>

#include "fused_body.cuh"

namespace spect {

namespace {

struct GroupPlan {
    Geometry g;
    FusedDims df, da;  // forward / adjoint launch shapes
    int cls_z;
    const float* rtab;
    const float* xt;
    const float* mubar;
    float* slab;
    const float* fx;
    const float* fz;
    float* part;
    const float* fx_adj;
    const float* fz_adj;
    float* ratio;
    const float* y;
    const float* rbar;
    size_t nproj;
    int* err;
};
struct GroupPlans {
    GroupPlan p[kGroupMax];
    GroupGrid grid;
};

struct GroupT {
    const float* in;
    float* out;
    int R, C;
};
struct GroupTs {
    GroupT p[kGroupMax];
    GroupGrid grid;
};

template <int P, bool MUS>
__global__ void __launch_bounds__(kRotThreads, 2) k_rot_fwd_grp(const __grid_constant__ GroupPlans gp)
{
    const int4 w = group_item(gp.grid);
    const GroupPlan q = gp.p[w.x];  // by value: the fields live in registers, not re-read from parameter space
    rot_fwd_body<P, MUS>(q.g, q.df, q.rtab, q.xt, q.mubar, q.slab, 0, q.err, w.y, w.z);
}

template <int P, bool TILED>
__global__ void __launch_bounds__(kFusedThreads, 1) k_fwd_sep_grp(const __grid_constant__ GroupPlans gp)
{
    const int4 w = group_item(gp.grid);
    const GroupPlan q = gp.p[w.x];  // by value: the fields live in registers, not re-read from parameter space
    fwd_sep_body<P, TILED>(q.g, q.df, q.slab, q.fx, q.fz, q.part, 0, q.err, w.y, w.z, w.w);
}

template <int P, bool TILED>
__global__ void __launch_bounds__(kFusedThreads, 1) k_adj_sep_grp(const __grid_constant__ GroupPlans gp)
{
    const int4 w = group_item(gp.grid);
    const GroupPlan q = gp.p[w.x];  // by value: the fields live in registers, not re-read from parameter space
    adj_sep_body<P, TILED>(q.g, q.da, q.cls_z, q.ratio, q.mubar, q.fx_adj, q.fz_adj, q.slab, 0, q.err, w.y, w.z,
                           w.w);
}

// v = sum over depth groups (fixed order), then the EM ratio y / (v + rbar): k_fwd_reduce per plan
constexpr int kReduceThreads = 256;
__global__ void __launch_bounds__(kReduceThreads) k_fwd_reduce_grp(const __grid_constant__ GroupPlans gp)
{
    const int4 w = group_item(gp.grid);
    const GroupPlan q = gp.p[w.x];  // by value: the fields live in registers, not re-read from parameter space
    const size_t o = (size_t)w.y * kReduceThreads + threadIdx.x;
    if (o >= q.nproj) return;
    float s = 0.f;
    for (int gq = 0; gq < q.df.G; ++gq) s += q.part[(size_t)gq * q.nproj + o];
    const float yb = s + (q.rbar ? q.rbar[o] : 0.f);
    q.ratio[o] = yb > 0.f ? q.y[o] / yb : 0.f;
}

__global__ void k_transpose_grp(const __grid_constant__ GroupTs gt)
{
    const int4 w = group_item(gt.grid);
    const GroupT& q = gt.p[w.x];
    transpose_body(q.in, q.out, q.R, q.C, w.y, w.z);
}

size_t plan_work(const spect_plan_s* P)
{
    return (size_t)P->g.nx * P->g.ny * P->g.nz * P->g.nview;
}

// chunks of at most kGroupMax plan indices, largest plans first
std::vector<std::vector<int>> chunks_of(std::vector<int> idx, const std::vector<spect_plan_s*>& plans)
{
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return plan_work(plans[a]) > plan_work(plans[b]); });
    std::vector<std::vector<int>> out;
    for (size_t i = 0; i < idx.size(); i += kGroupMax)
        out.emplace_back(idx.begin() + i, idx.begin() + std::min(idx.size(), i + (size_t)kGroupMax));
    return out;
}

template <int P>
void fill_plan(GroupPlan& q, const spect_plan_s* Pl, const float* y, const float* rbar)
{
    q.g = Pl->g;
    q.df = dims_for<P>(Pl->g, Pl->fused_J, Pl->fused_nT);
    q.da = dims_for<P>(Pl->g, Pl->adj_J, Pl->fused_nT);
    q.cls_z = Pl->cls_z;
    q.rtab = Pl->rtab;
    q.xt = Pl->xt;
    q.mubar = Pl->mubar;
    q.slab = Pl->slab;
    q.fx = Pl->fx;
    q.fz = Pl->fz;
    q.part = Pl->part;
    q.fx_adj = Pl->fx_adj;
    q.fz_adj = Pl->fz_adj;
    q.ratio = Pl->ratio;
    q.y = y;
    q.rbar = rbar;
    q.nproj = (size_t)Pl->g.nx * Pl->g.nz * Pl->g.nview;
    q.err = Pl->err;
}

// the shared memory the rotation kernel takes for this plan, and whether the
// attenuation plane is staged (the choice rot_launch makes)
template <int P>
size_t rot_smem(const spect_plan_s& Pl, bool* mus)
{
    const FusedDims d = dims_for<P>(Pl.g, Pl.fused_J, Pl.fused_nT);
    const size_t smin = rot_smem_min(d);
    const size_t smem_mu = smin + (size_t)d.ps * sizeof(float) + 16;
    *mus = smem_mu <= (size_t)Pl.smem_optin;
    return *mus ? smem_mu : smin;
}

// append plan m's grid (gx x gy x gz blocks) to a grouped launch's block ranges
void add_grid(GroupGrid& gg, int m, int gx, int gy, int gz)
{
    if (m == 0) gg.first[0] = 0;
    gg.gx[m] = gx;
    gg.gy[m] = gy;
    gg.first[m + 1] = gg.first[m] + gx * gy * gz;
    gg.n = m + 1;
}

template <class K, class A>
GroupLaunch make_launch(K kern, const A& args, dim3 threads, size_t smem)
{
    const unsigned blocks = (unsigned)args.grid.first[args.grid.n];
    return [=](cudaStream_t st) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<blocks, threads, smem, st>>>(args);
        return cudaGetLastError();
    };
}

// the launches of one stage for the plans `idx` of bucket P
template <int P>
cudaError_t stage_launches(int stage, const std::vector<int>& idx, const std::vector<spect_plan_s*>& plans,
                           const float* const* y, const float* const* rbar, GroupedBatch& /*B*/,
                           std::vector<GroupLaunch>& out)
{
    // sub-groups by kernel variant: attenuation staged (rotation) / tiled (blurs)
    std::vector<int> var[2];
    for (int i : idx) {
        bool flag = false;
        if (stage == 0) rot_smem<P>(*plans[i], &flag);
        else flag = dims_for<P>(plans[i]->g, plans[i]->fused_J, plans[i]->fused_nT).nT > 1;
        var[flag ? 1 : 0].push_back(i);
    }
    for (int f = 0; f < 2; ++f) {
        for (const std::vector<int>& ch : chunks_of(var[f], plans)) {
            GroupPlans gp{};
            size_t smem = 0;
            for (int m = 0; m < (int)ch.size(); ++m) {
                const spect_plan_s* Pl = plans[ch[m]];
                fill_plan<P>(gp.p[m], Pl, y[ch[m]], rbar ? rbar[ch[m]] : nullptr);
                const GroupPlan& q = gp.p[m];
                if (stage == 0) {  // the rotation's grid: (plane j, view)
                    bool mus = false;
                    smem = std::max(smem, rot_smem<P>(*Pl, &mus));
                    add_grid(gp.grid, m, q.g.ny, q.g.nview, 1);
                } else {           // the blurs' grid: (depth group, view, column tile)
                    const FusedDims& d = stage == 1 ? q.df : q.da;
                    smem = std::max(smem, stage == 1 ? smem_fwd<P>(q.g, d) : smem_adj<P>(q.g, d));
                    add_grid(gp.grid, m, d.G, q.g.nview, d.nT);
                }
            }
            if (ch.empty()) continue;
            if (stage == 0)
                out.push_back(f ? make_launch(k_rot_fwd_grp<P, true>, gp, dim3(kRotThreads), smem)
                                : make_launch(k_rot_fwd_grp<P, false>, gp, dim3(kRotThreads), smem));
            else if (stage == 1)
                out.push_back(f ? make_launch(k_fwd_sep_grp<P, true>, gp, dim3(kFusedThreads), smem)
                                : make_launch(k_fwd_sep_grp<P, false>, gp, dim3(kFusedThreads), smem));
            else
                out.push_back(f ? make_launch(k_adj_sep_grp<P, true>, gp, dim3(kFusedThreads), smem)
                                : make_launch(k_adj_sep_grp<P, false>, gp, dim3(kFusedThreads), smem));
        }
    }
    return cudaSuccess;
}

cudaError_t stage_by_bucket(int stage, const std::vector<spect_plan_s*>& plans, const float* const* y,
                            const float* const* rbar, GroupedBatch& B, std::vector<GroupLaunch>& out)
{
    for (int b : kBuckets) {
        std::vector<int> idx;
        for (int i = 0; i < (int)plans.size(); ++i)
            if (plans[i]->bucket == b) idx.push_back(i);
        if (idx.empty()) continue;
        cudaError_t e = cudaErrorInvalidValue;
        switch (b) {
#define SPECT_GB(B_)                                                      \
    case B_: e = stage_launches<B_>(stage, idx, plans, y, rbar, B, out); \
        break;
            SPECT_GB(3) SPECT_GB(5) SPECT_GB(7) SPECT_GB(9) SPECT_GB(11) SPECT_GB(13) SPECT_GB(15) SPECT_GB(17)
            SPECT_GB(21) SPECT_GB(25) SPECT_GB(29) SPECT_GB(33) SPECT_GB(37)
#undef SPECT_GB
            default: break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// the depth-group reduce with the EM ratio, all plans (any bucket)
cudaError_t reduce_launches(const std::vector<spect_plan_s*>& plans, const float* const* y, const float* const* rbar,
                            GroupedBatch& /*B*/, std::vector<GroupLaunch>& out)
{
    std::vector<int> all(plans.size());
    std::iota(all.begin(), all.end(), 0);
    for (const std::vector<int>& ch : chunks_of(all, plans)) {
        GroupPlans gp{};
        for (int m = 0; m < (int)ch.size(); ++m) {
            const spect_plan_s* Pl = plans[ch[m]];
            GroupPlan& q = gp.p[m];
            q.g = Pl->g;
            q.df.G = fused_groups(*Pl);
            q.part = Pl->part;
            q.ratio = Pl->ratio;
            q.y = y[ch[m]];
            q.rbar = rbar ? rbar[ch[m]] : nullptr;
            q.nproj = (size_t)Pl->g.nx * Pl->g.nz * Pl->g.nview;
            add_grid(gp.grid, m, (int)((q.nproj + kReduceThreads - 1) / kReduceThreads), 1, 1);
        }
        out.push_back(make_launch(k_fwd_reduce_grp, gp, dim3(kReduceThreads), 0));
    }
    return cudaSuccess;
}

// x (image layout) <-> x_t ([j][i][k]) for every plan: to_internal / from_internal
cudaError_t transpose_launches(const std::vector<spect_plan_s*>& plans, float* const* x, bool to_internal,
                               GroupedBatch& /*B*/, std::vector<GroupLaunch>& out)
{
    std::vector<int> all(plans.size());
    std::iota(all.begin(), all.end(), 0);
    for (const std::vector<int>& ch : chunks_of(all, plans)) {
        GroupTs gt{};
        for (int m = 0; m < (int)ch.size(); ++m) {
            const spect_plan_s* Pl = plans[ch[m]];
            const int nxy = Pl->g.nx * Pl->g.ny, nz = Pl->g.nz;
            GroupT& q = gt.p[m];
            q.in = to_internal ? x[ch[m]] : Pl->xt;
            q.out = to_internal ? Pl->xt : x[ch[m]];
            q.R = to_internal ? nz : nxy;
            q.C = to_internal ? nxy : nz;
            add_grid(gt.grid, m, (q.C + 31) / 32, (q.R + 31) / 32, 1);
        }
        out.push_back(make_launch(k_transpose_grp, gt, dim3(32, 8), 0));
    }
    return cudaSuccess;
}

}  // namespace

bool groupable(const spect_plan_s& P)
{
    return P.fast && P.separable && !P.rot3 && !P.recompute && P.gather && P.bucket > 0 && P.chunk >= P.g.nview &&
           P.adj_chunk >= P.g.nview;
}

cudaError_t build_grouped(const std::vector<spect_plan_s*>& plans, float* const* x, const float* const* y,
                          const float* const* rbar, GroupedBatch& B)
{
    cudaError_t e = transpose_launches(plans, x, true, B, B.head);
    if (e == cudaSuccess) e = stage_by_bucket(0, plans, y, rbar, B, B.iter);
    if (e == cudaSuccess) e = stage_by_bucket(1, plans, y, rbar, B, B.iter);
    if (e == cudaSuccess) e = reduce_launches(plans, y, rbar, B, B.iter);
    if (e == cudaSuccess) e = stage_by_bucket(2, plans, y, rbar, B, B.iter);
    if (e == cudaSuccess) e = build_grouped_gather(plans, B, B.iter);
    if (e == cudaSuccess) e = transpose_launches(plans, const_cast<float* const*>(x), false, B, B.tail);
    return e;
}

void free_grouped(GroupedBatch& B)
{
    B.head.clear();
    B.iter.clear();
    B.tail.clear();
}

}  // namespace spect
