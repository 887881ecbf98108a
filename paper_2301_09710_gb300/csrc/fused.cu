// fused.cu -- the default (fast) path of the projector on sm_103a.
//
// Same operator as the kernels in rotate.cu / conv.cu (Section II-A of
// arXiv 2301.09710, Algorithms 1 and 2), organised for GB300:
//
//  * Internal volumes use a k-fastest layout [j][i][k] ("transposed"): the
//    bilinear rotation weights depend on (i, j, view) only, so each of the four
//    neighbours of a rotated sample is a contiguous run of nz floats and every
//    rotation gather is a coalesced 128-byte access with lanes over k.
//  * The Eq. (1) attenuation factor mubar is computed once per plan for every
//    view, [l][j][i][k] (nview * nx*ny*nz floats; HBM is plentiful), so the hot
//    kernels multiply by a streamed, coalesced value instead of re-rotating mu.
//  * Forward: a rotation kernel rotates and attenuates every (view, depth)
//    plane into the work slab, already laid out as the blur kernel's shared-
//    memory image (replicate halo columns, conflict-free pitch).  The blur
//    kernel (one block per view and group of J depth planes) streams those
//    images in by TMA, runs the separable PSF blur as two register-blocked
//    sliding-window passes (i, then k; replicate padding along k folded into
//    edge taps), and accumulates the group's depth sum in shared memory; the
//    groups' partials are added in a fixed order by a small reduce kernel
//    (deterministic, no atomics).
//  * Transpose: one block per (view, depth group) expands the detector plane
//    into blurred-adjoint planes times mubar (the t slab, [v][j][i][k]); a
//    gather kernel then sums sum_l sum_p W_l(p;q) t_l(p,k) per destination voxel
//    q over fixed-length adjacency lists (weights bitwise those of A).
#include <algorithm>

#include "fused_body.cuh"

namespace spect {


// ============================================================================
// Plan-time kernels
// ============================================================================

// out[c][r] = in[r][c] for an R x C matrix (tiled through shared memory).
__global__ void k_transpose(const float* __restrict__ in, float* __restrict__ out, int R, int C)
{
    transpose_body(in, out, R, C, blockIdx.x, blockIdx.y);
}

cudaError_t launch_transpose(const float* in, float* out, int R, int C, cudaStream_t st)
{
    dim3 grid((C + 31) / 32, (R + 31) / 32);
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, out, R, C);
    return cudaGetLastError();
}

// mubar[l][j][i][k] = exp(-dy (mu~(j)/2 + sum_{s>j} mu~(s))), Eq. (1), for every
// view.  One block per (row i, view l = l0 + v, run of up to kMuThreads columns k):
// the block first stages the rotation-table entries of row i for every depth
// (the forward rotation's bilinear weights and base voxels) in shared memory,
// then each thread walks one column k from the detector side with a
// compensated running sum (AttenScan).  Lanes run over k, so the corner loads
// and the stores are coalesced, and a depth step's loads depend on nothing
// but the staged table, so the unrolled walk keeps several steps in flight.
// With nview * nx * nz independent columns this does O(1) work per factor; a
// warp scan along depth (atten_warp_scan) would do O(log 32) and measured
// 2.6x slower here.  mu_t is mu in the [j][i][k] layout; planes (l, j) are ps
// floats apart (16-byte aligned for bulk copies); view l lands at position v.
constexpr int kMuThreads = 128;

__global__ void __launch_bounds__(kMuThreads) k_mubar_cache(Geometry g, int ps, int ts,
                                                            const float* __restrict__ rtab,
                                                            const float* __restrict__ mu_t,
                                                            float* __restrict__ mubar, int l0)
{
    extern __shared__ __align__(16) float smu[];
    float4* TW = reinterpret_cast<float4*>(smu);        // [ny] weights of row i
    int* TB = reinterpret_cast<int*>(smu + 4 * g.ny);   // [ny] base voxels of row i
    const int k = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y, v = blockIdx.z, l = l0 + v;
    const float* tab_l = rtab + (size_t)l * g.ny * ts;
    for (int j = threadIdx.x; j < g.ny; j += blockDim.x) {
        const float* tab = tab_l + (size_t)j * ts;
        TW[j] = __ldg(reinterpret_cast<const float4*>(tab) + i);
        TB[j] = __ldg(reinterpret_cast<const int*>(tab + 4 * g.nx) + i);
    }
    __syncthreads();
    if (k >= g.nz) return;
    const size_t rs = (size_t)g.nx * g.nz;
    float* out = mubar + (size_t)v * g.ny * ps + (size_t)i * g.nz + k;
    if (!g.has_mu) {
        for (int j = 0; j < g.ny; ++j) out[(size_t)j * ps] = 1.f;
        return;
    }
    AttenScan sc;
#pragma unroll 8
    for (int j = g.ny - 1; j >= 0; --j) {
        const float4 w = TW[j];
        const float* m = mu_t + (size_t)TB[j] * g.nz + k;
        float mv = 0.f;
        mv = __fmaf_rn(w.x, __ldg(m), mv);
        mv = __fmaf_rn(w.y, __ldg(m + g.nz), mv);
        mv = __fmaf_rn(w.z, __ldg(m + rs), mv);
        mv = __fmaf_rn(w.w, __ldg(m + rs + g.nz), mv);
        out[(size_t)j * ps] = sc.step(mv, g.dy);
    }
}

namespace {
cudaError_t mubar_launch(const spect_plan_s& P, const float* mu_t, int l0, int nv, cudaStream_t st)
{
    const size_t smem = (size_t)P.g.ny * 5 * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_mubar_cache, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // a run of columns k per block: nz rounded up to whole warps, at most kMuThreads
    const int thr = std::min(kMuThreads, (P.g.nz + 31) & ~31);
    const dim3 grid((P.g.nz + thr - 1) / thr, P.g.nx, nv);
    k_mubar_cache<<<grid, thr, smem, st>>>(P.g, P.ps, P.ts, P.rtab, mu_t, P.mubar, l0);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_mubar_cache(const spect_plan_s& P, const float* mu_t, cudaStream_t st)
{
    return mubar_launch(P, mu_t, 0, P.g.nview, st);
}

cudaError_t launch_mubar_range(const spect_plan_s& P, int l0, int nv, cudaStream_t st)
{
    if (!P.recompute || !P.mut || nv < 1 || (size_t)nv * P.g.ny * P.ps > P.mubar_cap) return cudaErrorInvalidValue;
    return mubar_launch(P, P.mut, l0, nv, st);
}

// Rotation tables of every (view, depth row), the per-plane input of the fused
// forward: block (l, j) holds nx float4 weights then nx int bases (ts floats,
// 16-byte aligned), fetched together with the attenuation plane by one TMA
// transaction.
__global__ void k_rot_tables(Geometry g, int ts, const ViewRot* __restrict__ rot, float* __restrict__ tab)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)g.nview * g.ny * g.nx) return;
    const int i = (int)(idx % g.nx);
    const size_t lj = idx / g.nx;
    const int j = (int)(lj % g.ny), l = (int)(lj / g.ny);
    float4 w;
    int base;
    rot_table_entry(i, j, rot[l], g, w, base);
    float* blk = tab + lj * ts;
    reinterpret_cast<float4*>(blk)[i] = w;
    reinterpret_cast<int*>(blk + 4 * g.nx)[i] = base;
}

cudaError_t launch_rot_tables(const spect_plan_s& P, cudaStream_t st)
{
    const size_t n = (size_t)P.g.nview * P.g.ny * P.g.nx;
    k_rot_tables<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P.g, P.ts, P.rot, P.rtab);
    return cudaGetLastError();
}

// Fixed-length adjacency lists for the transposed rotation: for destination
// q and view l, up to `maxe` (source column offset j*ps + i*nz, weight) pairs,
// zero-padded, laid out [q][l][e].  The candidate search and weights are those
// of k_build_adjacency (rotate.cu).
__global__ void k_build_adjacency_fixed(Geometry g, int ps, const ViewRot* __restrict__ rot, int maxe, AdjEntry* adj)
{
    const size_t nxy = (size_t)g.nx * g.ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nxy * g.nview) return;
    const int l = (int)(idx / nxy);
    const int q = (int)(idx % nxy);
    const int qi = q % g.nx, qj = q / g.nx;
    const ViewRot r = rot[l];
    const float ct = r.ct_hi + r.ct_lo, st = r.st_hi + r.st_lo;
    const float c = (float)g.cint + g.cfrac;
    const float dqi = (float)qi - c, dqj = (float)qj - c;
    const float pi_ = c + ct * dqi - st * dqj;
    const float pj_ = c + st * dqi + ct * dqj;
    const int bi = (int)floorf(pi_) - 1, bj = (int)floorf(pj_) - 1;
    AdjEntry* out = adj + ((size_t)q * g.nview + l) * maxe;
    int cnt = 0;
    for (int cj = 0; cj < 4; ++cj)
        for (int ci = 0; ci < 4; ++ci) {
            const int pi = bi + ci, pj = bj + cj;
            if (pi < 0 || pi >= g.nx || pj < 0 || pj >= g.ny) continue;
            const Sample s = rot_sample(pi, pj, r, g.cint, g.cfrac);
            const int di = qi - s.i0, dj = qj - s.j0;
            if (di < 0 || di > 1 || dj < 0 || dj > 1) continue;
            const float w = bilinear_w(s, di, dj);
            if (w == 0.f || cnt >= maxe) continue;
            AdjEntry e;
            e.p = pj * ps + pi * g.nz;  // offset of the source column in a [j][i][k] slab with plane stride ps
            e.w = w;
            out[cnt++] = e;
        }
    for (; cnt < maxe; ++cnt) {
        AdjEntry e;
        e.p = 0;
        e.w = 0.f;
        out[cnt] = e;
    }
}

cudaError_t launch_build_adjacency_fixed(const spect_plan_s& P, cudaStream_t st)
{
    const size_t n = (size_t)P.g.nx * P.g.ny * P.g.nview;
    k_build_adjacency_fixed<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P.g, P.ps, P.rot, P.adj_max, P.adjf);
    return cudaGetLastError();
}

template <int P, bool MUS>
__global__ void __launch_bounds__(kRotThreads, 2) k_rot_fwd(Geometry g, FusedDims d, const float* __restrict__ rtab,
                                                         const float* __restrict__ xt,
                                                         const float* __restrict__ mubar, float* __restrict__ wsl,
                                                         int l0, int* err)
{
    rot_fwd_body<P, MUS>(g, d, rtab, xt, mubar, wsl, l0, err, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------
// Forward rotation with the three-pass rotation (rot3.cu): the same block, plane
// image, attenuation and output as k_rot_fwd, but every output (i, k) of plane
// j is the eight-tap sum  sum_m w_m x_t[off_m + k]  of its table row (the three
// passes' products; unused taps have weight 0, offset 0).  The (view, row)
// table -- nx x 8 weights, then nx x 8 offsets -- is staged in shared memory
// once; warps take one row i per step with lanes over k (24 gathers in
// flight per lane, as k_rot_fwd's row pairs).
// ----------------------------------------------------------------------------
template <int P, bool MUS>
__global__ void __launch_bounds__(kRotThreads, 2) k_rot_fwd8(Geometry g, FusedDims d, const float* __restrict__ tab8,
                                                          const float* __restrict__ xt,
                                                          const float* __restrict__ mubar, float* __restrict__ wsl,
                                                          int l0, int* err)
{
    constexpr int C = Sep<P>::C;
    extern __shared__ __align__(16) float sm[];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int ts8 = 16 * nx;
    float* S = sm;
    float* TBL = sm + d.farea;  // nx x 8 weights, then nx x 8 int offsets
    float* MU = TBL + ts8;      // [i][k] attenuation plane (MUS)
    uint64_t* bar = reinterpret_cast<uint64_t*>(MU + d.ps);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = kRotThreads / 32;
    const int j = blockIdx.x, v = blockIdx.y, l = l0 + v;
    const int wp = d.wpf;
    const int wcols = d.nib * Sep<P>::CX + 2 * C;
    const float* tab = tab8 + ((size_t)l * ny + j) * ts8;
    const float* mb = mubar + ((size_t)l * ny + j) * d.ps;
    if (MUS && threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_load_1d(MU, mb, (unsigned)d.ps * 4u, bar);
    }
    for (int e = threadIdx.x; e < ts8 / 4; e += kRotThreads)
        reinterpret_cast<float4*>(TBL)[e] = __ldg(reinterpret_cast<const float4*>(tab) + e);
    __syncthreads();  // table staged; the barrier is initialised before anyone waits on it
    const int* OFF = reinterpret_cast<const int*>(TBL + 8 * nx);
    bool ok = true, waited = !MUS;

    for (int i = warp; i < nx; i += NW) {
        const float4 wl = reinterpret_cast<const float4*>(TBL)[2 * i];
        const float4 wh = reinterpret_cast<const float4*>(TBL)[2 * i + 1];
        const int4 ol = reinterpret_cast<const int4*>(OFF)[2 * i];
        const int4 oh = reinterpret_cast<const int4*>(OFF)[2 * i + 1];
        const float w[8] = {wl.x, wl.y, wl.z, wl.w, wh.x, wh.y, wh.z, wh.w};
        const int o[8] = {ol.x, ol.y, ol.z, ol.w, oh.x, oh.y, oh.z, oh.w};
        for (int k0 = 0; k0 < nz; k0 += 96) {
            float xs[3][8], ma[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int k = k0 + 32 * q + lane;
                if (k < nz) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) xs[q][m] = __ldg(xt + o[m] + k);
                    if (!MUS) ma[q] = __ldg(mb + i * nz + k);
                }
            }
            if (!waited) {
                ok = mbar_wait_bounded(bar, 0u);
                waited = true;
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int k = k0 + 32 * q + lane;
                if (k < nz) {
                    if (MUS) ma[q] = MU[i * nz + k];
                    float* wr = S + k * wp + C;
                    float va = w[0] * xs[q][0];
#pragma unroll
                    for (int m = 1; m < 8; ++m) va = fmaf(w[m], xs[q][m], va);
                    va *= ma[q];
                    wr[i] = va;
                    if (i == 0)  // replicate padding along i: left halo columns
                        for (int h = -C; h < 0; ++h) wr[h] = va;
                    if (i == nx - 1)  // right halo columns
                        for (int h = nx; h < wcols - C; ++h) wr[h] = va;
                }
            }
        }
    }
    if (__syncthreads_or(!ok)) {  // the attenuation plane never arrived
        if (threadIdx.x == 0) {
            flag_timeout(err);
            mbar_wait_bounded(bar, 0u);  // a last chance for the copy in flight to land
        }
        return;
    }
    float* dst = wsl + ((size_t)v * ny + j) * d.parea;
    if (d.nT == 1) {
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            tma_store_1d(dst, S, (unsigned)d.parea * 4u);
            tma_store_wait_read<0>();  // the block may leave once its shared memory is read
        }
        return;
    }
    for (int r = warp; r < d.nT * nz; r += NW) {
        const int t = r / nz, k = r - t * nz;
        const int tw = min(d.TI + 2 * C, wcols - t * d.TI);
        const float* src = S + k * wp + t * d.TI;
        float* out = dst + (size_t)t * d.warea + (size_t)k * d.wp;
        for (int c = lane; c < tw; c += 32) out[c] = src[c];
    }
}

// ----------------------------------------------------------------------------
// Forward blur + depth sum: one block per (depth group of J planes, view,
// column tile).
// Rotated planes arrive by TMA into a double buffer (plane j+2 is requested as
// soon as plane j's i-pass has read its buffer); per plane the i-pass writes U
// (k halos by warp shuffles), the k-pass accumulates into ACC.
// ----------------------------------------------------------------------------
template <int P, bool TILED>
__global__ void __launch_bounds__(kFusedThreads, 1) k_fwd_sep_fused(Geometry g, FusedDims d,
                                                                     const float* __restrict__ wsl,
                                                                     const float* __restrict__ fx,
                                                                     const float* __restrict__ fz,
                                                                     float* __restrict__ part, int l0, int* err)
{
    fwd_sep_body<P, TILED>(g, d, wsl, fx, fz, part, l0, err, blockIdx.x, blockIdx.y, blockIdx.z);
}

// v(i,k,l) = sum over depth groups of the partials (fixed order), optionally
// turned into the EM ratio y / (v + rbar).
__global__ void k_fwd_reduce(const float* __restrict__ part, int G, size_t nproj, float* __restrict__ v,
                             const float* __restrict__ em_y, const float* __restrict__ em_rbar)
{
    const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nproj) return;
    float s = 0.f;
    for (int gq = 0; gq < G; ++gq) s += part[(size_t)gq * nproj + o];
    if (em_y) {
        const float yb = s + (em_rbar ? em_rbar[o] : 0.f);
        v[o] = yb > 0.f ? em_y[o] / yb : 0.f;
    } else {
        v[o] = s;
    }
}

template <int P, bool TILED>
__global__ void __launch_bounds__(kFusedThreads, 1) k_adj_sep_fused(Geometry g, FusedDims d, int cls_z,
                                                                     const float* __restrict__ vin,
                                                                     const float* __restrict__ mubar,
                                                                     const float* __restrict__ fx_adj,
                                                                     const float* __restrict__ fz_adj,
                                                                     float* __restrict__ slab, int l0, int* err)
{
    adj_sep_body<P, TILED>(g, d, cls_z, vin, mubar, fx_adj, fz_adj, slab, l0, err, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ============================================================================
// Fused blur for a full (non-separable) PSF p(a, b, j, l), padded tap count P.
// The 2D convolution of a plane is a sum over tap rows b of 1D FIRs along i
// (taps p(:, b)) applied to row k - b + cz: every term of a row runs through
// the register-blocked FIR of the separable kernels, and the rows add up per
// output (a row partial per b, then the sum over b: short FP32 chains).
//   forward: the rotated planes come from k_rot_fwd (same images as the
//     separable path: W[k][C + i] with replicate halo columns); ZH replicate
//     halo rows above and below are filled in shared memory after each TMA
//     load; outputs accumulate over the group's planes in ACC[i][k].
//   adjoint: the detector plane is staged once per block, zero-padded
//     (Vx[ZH + k][C + i]); per plane the taps of the k edge class of each
//     output row are used for the whole run, and the first / last detector
//     column (the i edge classes) is recomputed with its own variant.
// ============================================================================
__host__ __device__ inline int dir_rows(int nz, int ZH) { return nz + 2 * ZH; }

__host__ __device__ inline size_t dir_fwd_smem_floats(const FusedDims& d, int nz, int P, int PT, int ZH)
{
    const size_t xarea = ((size_t)dir_rows(nz, ZH) * d.wp + 3) & ~(size_t)3;
    // Wext x2 | taps P x PT | ACC | 2 mbarriers
    return 2 * xarea + (size_t)P * PT + (size_t)d.urows * d.apc + 8;
}

__host__ __device__ inline size_t dir_adj_smem_floats(const FusedDims& d, int nz, int P, int PT, int ZH, int ncls)
{
    const size_t xarea = ((size_t)dir_rows(nz, ZH) * d.wp + 3) & ~(size_t)3;
    // Vx | MB x2 | taps ncls x P x PT | 2 mbarriers
    return xarea + 2 * (size_t)d.marea + (size_t)ncls * P * PT + 8;
}

template <int P>
__global__ void __launch_bounds__(kFusedThreads, 1) k_fwd_dir_fused(Geometry g, FusedDims d,
                                                                     const float* __restrict__ wsl,
                                                                     const float* __restrict__ psf,
                                                                     float* __restrict__ part, int l0, int* err)
{
    using S = Sep<P>;
    constexpr int C = S::C, CX = S::CX, ZH = S::ZH, PT = S::PT;
    extern __shared__ __align__(16) float sm[];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int xarea = (dir_rows(nz, ZH) * d.wp + 3) & ~3;
    float* WB = sm;                                 // [2][xarea]: rows -ZH .. nz+ZH-1 of a plane image
    float* TAP = WB + 2 * (size_t)xarea;            // [P][PT], this plane's taps (zero-padded, centred)
    float* ACC = TAP + (size_t)P * PT;              // [i][k], apc pitch
    uint64_t* bar = reinterpret_cast<uint64_t*>(ACC + (size_t)d.urows * d.apc);
    const int tid = threadIdx.x;
    constexpr int T = kFusedThreads;
    const int grp = blockIdx.x, v = blockIdx.y, l = l0 + v;
    const int lp = g.nvp == 1 ? 0 : l;
    const int j_begin = grp * d.J, j_end = min(ny, j_begin + d.J);
    const int ox = (P - g.px) / 2, oz = (P - g.pz) / 2;
    const int pln = nx * nz;
    const float* wv = wsl + (size_t)v * ny * d.parea;

    for (int e = tid; e < d.urows * d.apc; e += T) ACC[e] = 0.f;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_load_1d(WB + ZH * d.wp, wv + (size_t)j_begin * d.parea, (unsigned)d.warea * 4u, bar);
        if (j_begin + 1 < j_end)
            tma_load_1d(WB + xarea + ZH * d.wp, wv + (size_t)(j_begin + 1) * d.parea, (unsigned)d.warea * 4u,
                        bar + 1);
    }
    __syncthreads();

    unsigned phases = 0u;
    for (int j = j_begin; j < j_end; ++j) {
        const int b = (j - j_begin) & 1;
        float* W = WB + b * (size_t)xarea;
        const bool ok = mbar_wait_bounded(bar + b, (phases >> b) & 1u);
        phases ^= 1u << b;
        // this plane's taps, and the replicate halo rows (copies of rows 0 and nz-1)
        const float* pp = psf + ((size_t)lp * ny + j) * g.px * g.pz;
        for (int e = tid; e < P * PT; e += T) {
            const int bb = e / PT, a = e - bb * PT, ax = a - ox, bz = bb - oz;
            TAP[e] = (ax >= 0 && ax < g.px && bz >= 0 && bz < g.pz) ? __ldg(pp + (size_t)bz * g.px + ax) : 0.f;
        }
        if (ok)
            for (int e = tid; e < 2 * C * d.wp; e += T) {
                const int r = e / d.wp, c = e - r * d.wp;
                if (r < C) W[(ZH - C + r) * d.wp + c] = W[ZH * d.wp + c];
                else W[(ZH + nz + r - C) * d.wp + c] = W[(ZH + nz - 1) * d.wp + c];
            }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                flag_timeout(err);
                mbar_wait_bounded(bar + b, ((phases >> b) & 1u) ^ 1u);
                mbar_wait_bounded(bar + (b ^ 1), (phases >> (b ^ 1)) & 1u);
            }
            return;
        }
        // c_j(i, k) = sum_b FIR_i(taps p(:, b), row k - b + cz); lanes over k
        for (int it = tid; it < nz * d.nib; it += T) {
            const int ib = it / nz, k = it - ib * nz;
            const int li = ib * CX;
            float o[CX];
#pragma unroll
            for (int c = 0; c < CX; ++c) o[c] = 0.f;
            for (int bb = 0; bb < P; ++bb) {
                const float* wr = W + (ZH + k - bb + C) * d.wp + li;
                float win[4 * ((CX + P - 1 + 3) / 4)];
                load_row_f4(wr, win);
                float ob[CX];
                fir<P, CX, -1, P - 1>(TAP + bb * PT, win, ob);
#pragma unroll
                for (int c = 0; c < CX; ++c) o[c] += ob[c];
            }
            float* ac = ACC + li * d.apc + k;
            if (li + CX <= nx) {
#pragma unroll
                for (int c = 0; c < CX; ++c) ac[c * d.apc] += o[c];
            } else {
#pragma unroll
                for (int c = 0; c < CX; ++c)
                    if (li + c < nx) ac[c * d.apc] += o[c];
            }
        }
        __syncthreads();  // buffer b and the taps are free
        if (tid == 0 && j + 2 < j_end) {
            fence_proxy_async_smem();
            tma_load_1d(W + ZH * d.wp, wv + (size_t)(j + 2) * d.parea, (unsigned)d.warea * 4u, bar + b);
        }
    }
    float* pout = part + ((size_t)grp * g.nview + l) * pln;
    for (int e = tid; e < pln; e += T) {
        const int k = e / nx, i = e - k * nx;
        pout[e] = ACC[i * d.apc + k];
    }
}

template <int P>
__global__ void __launch_bounds__(kFusedThreads, 1) k_adj_dir_fused(Geometry g, FusedDims d, int cls_z,
                                                                     const float* __restrict__ vin,
                                                                     const float* __restrict__ mubar,
                                                                     const float* __restrict__ psf_adj,
                                                                     float* __restrict__ slab, int l0, int* err)
{
    using S = Sep<P>;
    constexpr int C = S::C, CX = S::CX, ZH = S::ZH, PT = S::PT;
    extern __shared__ __align__(16) float sm[];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int xarea = (dir_rows(nz, ZH) * d.wp + 3) & ~3;
    const int ncls = 3 * cls_z;                    // edge classes (ci, ck)
    float* Vx = sm;                                // zero-padded detector plane, Vx[ZH + k][C + i]
    float* MB = Vx + xarea;                        // [2][marea]
    float* TAP = MB + 2 * (size_t)d.marea;         // [ci * cls_z + ck][P][PT], this plane
    uint64_t* bar = reinterpret_cast<uint64_t*>(TAP + (size_t)ncls * P * PT);
    const int tid = threadIdx.x;
    constexpr int T = kFusedThreads;
    const int grp = blockIdx.x, v = blockIdx.y, l = l0 + v;
    const int lp = g.nvp == 1 ? 0 : l;
    const int j_begin = grp * d.J, j_end = min(ny, j_begin + d.J);
    const int ox = (P - g.px) / 2, oz = (P - g.pz) / 2;
    const size_t nrow = (size_t)g.nvp * ny, pplane = (size_t)g.px * g.pz;
    const int pln = nx * nz;
    const float* mub = mubar + ((size_t)l * ny) * d.ps;
    float* tsl = slab + ((size_t)v * ny) * d.ps;
    const unsigned mbytes = (unsigned)d.ps * 4u;

    for (int e = tid; e < xarea; e += T) Vx[e] = 0.f;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_load_1d(MB, mub + (size_t)j_begin * d.ps, mbytes, bar);
    }
    __syncthreads();
    for (int e = tid; e < pln; e += T) {
        const int k = e / nx, i = e - k * nx;
        Vx[(ZH + k) * d.wp + C + i] = vin[(size_t)l * pln + e];
    }

    unsigned phases = 0u;
    for (int j = j_begin; j < j_end; ++j) {
        const int b = (j - j_begin) & 1;
        // taps of every edge class of this plane
        for (int e = tid; e < ncls * P * PT; e += T) {
            const int cls = e / (P * PT), r = e - cls * P * PT, bb = r / PT, a = r - bb * PT;
            const int ax = a - ox, bz = bb - oz;
            TAP[e] = (ax >= 0 && ax < g.px && bz >= 0 && bz < g.pz)
                         ? __ldg(psf_adj + ((size_t)cls * nrow + (size_t)lp * ny + j) * pplane + (size_t)bz * g.px + ax)
                         : 0.f;
        }
        __syncthreads();
        // the other buffer receives the next plane's attenuation once its store has read it
        if (tid == 0 && j + 1 < j_end) {
            tma_store_wait_read<0>();
            tma_load_1d(MB + (b ^ 1) * (size_t)d.marea, mub + (size_t)(j + 1) * d.ps, mbytes, bar + (b ^ 1));
        }
        float* mb = MB + b * (size_t)d.marea;
        const bool ok = mbar_wait_bounded(bar + b, (phases >> b) & 1u);
        phases ^= 1u << b;
        if (ok) {
            for (int it = tid; it < nz * d.nib; it += T) {
                const int ib = it / nz, k = it - ib * nz;
                const int li = ib * CX;
                const int ck = nz == 1 ? 0 : (k == 0 ? 1 : (k == nz - 1 ? 2 : 0));
                const float* TK = TAP + (size_t)ck * P * PT;  // class (ci = interior, ck)
                float o[CX];
#pragma unroll
                for (int c = 0; c < CX; ++c) o[c] = 0.f;
                for (int bb = 0; bb < P; ++bb) {
                    const float* vr = Vx + (ZH + k + bb - C) * d.wp + li;
                    float win[4 * ((CX + P - 1 + 3) / 4)];
                    load_row_f4(vr, win);
                    float ob[CX];
                    fir<P, CX, 1, 0>(TK + bb * PT, win, ob);
#pragma unroll
                    for (int c = 0; c < CX; ++c) o[c] += ob[c];
                }
                // first / last detector column: their own edge-class variant
                const int cl = nx - 1 - li;
                if (li == 0 || cl < CX) {
                    auto edge = [&](int c, int ci) {
                        const float* TC = TAP + (size_t)(ci * cls_z + ck) * P * PT;
                        float acc = 0.f;
#pragma unroll 2
                        for (int bb = 0; bb < P; ++bb) {
                            const float* vr = Vx + (ZH + k + bb - C) * d.wp + li + c;
                            float rp = 0.f;
#pragma unroll
                            for (int a = 0; a < P; ++a) rp = fmaf(TC[bb * PT + a], vr[a], rp);
                            acc += rp;
                        }
                        return acc;
                    };
                    if (li == 0) o[0] = edge(0, 1);
                    if (cl < CX) {
#pragma unroll
                        for (int c = 0; c < CX; ++c)
                            if (c == cl) o[c] = edge(c, nx == 1 ? 0 : 2);
                    }
                }
                float* mp = mb + li * nz + k;
#pragma unroll
                for (int c = 0; c < CX; ++c)
                    if (li + c < nx) mp[c * nz] = o[c] * mp[c * nz];
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                flag_timeout(err);
                mbar_wait_bounded(bar + b, ((phases >> b) & 1u) ^ 1u);
                tma_store_wait_all();
            }
            return;
        }
        if (tid == 0) {
            fence_proxy_async_smem();
            tma_store_1d(tsl + (size_t)j * d.ps, mb, mbytes);
        }
    }
    if (tid == 0) tma_store_wait_read<0>();  // the writes complete with the grid
}

// x_t(q,k) (+)= sum_{v in chunk} sum_{e < MAXE} w_e t[v][p_e][k]
// with the EM update (em_update) on the last chunk when em.x is set.  The
// lists are laid out [q][l][e] so one destination's entries for all views are
// contiguous; each entry holds the premultiplied offset p*nz of its source
// column in the slab.  A thread owns VEC consecutive k of one destination (float4 loads
// when nz % 4 == 0).  Per view the few terms are summed plainly, the views
// with Kahan compensation.
template <int VEC>
struct VecT;
template <>
struct VecT<1> {
    using type = float;
};
template <>
struct VecT<4> {
    using type = float4;
};

template <int MAXE, int VEC>
__global__ void __launch_bounds__(256) k_adj_rot_t(Geometry g, int ps, const AdjEntry* __restrict__ adj,
                                                   const float* __restrict__ slab, int l0, int nv, float* out,
                                                   int accumulate, EmArgs em)
{
    using VT = typename VecT<VEC>::type;
    const int nxy = g.nx * g.ny;
    const int nzv = g.nz / VEC;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nxy * nzv) return;
    const int qq = idx / nzv;
    const int k = (idx - qq * nzv) * VEC;
    // destinations in strips 4 wide in i running along j: a block covers a
    // compact patch, so the ~4 reads of each source column mostly hit L1
    int q = qq;
    if ((g.nx & 3) == 0) {
        const int strip = qq / (4 * g.ny), r = qq - strip * 4 * g.ny;
        q = (4 * strip + (r & 3)) + g.nx * (r >> 2);
    }
    const AdjEntry* e = adj + ((size_t)q * g.nview + l0) * MAXE;
    const float* t = slab + k;
    const size_t vstride = (size_t)g.ny * ps;
    KSum acc[VEC];
    // four views per step: all entry loads, then all slab loads, are issued
    // before any is used, so the chain of dependent loads is 4x shorter
    constexpr int UV = 4;
    int v = 0;
    for (; v + UV <= nv; v += UV) {
        AdjEntry a[UV][MAXE];
#pragma unroll
        for (int w = 0; w < UV; ++w)
#pragma unroll
            for (int m = 0; m < MAXE; ++m) a[w][m] = e[w * MAXE + m];
        VT tv[UV][MAXE];
#pragma unroll
        for (int w = 0; w < UV; ++w)
#pragma unroll
            for (int m = 0; m < MAXE; ++m) tv[w][m] = *reinterpret_cast<const VT*>(t + w * vstride + a[w][m].p);
#pragma unroll
        for (int w = 0; w < UV; ++w) {
            float sv[VEC];
#pragma unroll
            for (int u = 0; u < VEC; ++u) sv[u] = 0.f;
#pragma unroll
            for (int m = 0; m < MAXE; ++m) {
                const float* tf = reinterpret_cast<const float*>(&tv[w][m]);
#pragma unroll
                for (int u = 0; u < VEC; ++u) sv[u] = fmaf(a[w][m].w, tf[u], sv[u]);
            }
#pragma unroll
            for (int u = 0; u < VEC; ++u) acc[u].add(sv[u]);
        }
        e += UV * MAXE;
        t += UV * vstride;
    }
    for (; v < nv; ++v) {
        AdjEntry a[MAXE];
#pragma unroll
        for (int m = 0; m < MAXE; ++m) a[m] = e[m];
        VT tv[MAXE];
#pragma unroll
        for (int m = 0; m < MAXE; ++m) tv[m] = *reinterpret_cast<const VT*>(t + a[m].p);
        float sv[VEC];
#pragma unroll
        for (int u = 0; u < VEC; ++u) sv[u] = 0.f;
#pragma unroll
        for (int m = 0; m < MAXE; ++m) {
            const float* tf = reinterpret_cast<const float*>(&tv[m]);
#pragma unroll
            for (int u = 0; u < VEC; ++u) sv[u] = fmaf(a[m].w, tf[u], sv[u]);
        }
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[u].add(sv[u]);
        e += MAXE;
        t += vstride;
    }
    const size_t o = (size_t)q * g.nz + k;
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
        float val = acc[u].value();
        if (accumulate) val += out[o + u];
        if (em.x) em.x[o + u] = em_update(em.x[o + u], val, em.s[o + u], em.u ? em.u[o + u] : 0.f, em.beta);
        else out[o + u] = val;
    }
}

// ============================================================================
// host side: dimensioning and launchers
// ============================================================================
namespace {
template <int P>
int tiles_that_fit(const Geometry& g, size_t limit, int min_tiles)
{
    const int nib = (g.nx + Sep<P>::CX - 1) / Sep<P>::CX;
    int last_nt = 0;
    for (int t = min_tiles < 1 ? 1 : min_tiles; t <= nib; ++t) {
        const FusedDims d = dims_for<P>(g, 8, t);
        if (d.nT == last_nt) continue;  // same tile width as a smaller request
        last_nt = d.nT;
        if (smem_fwd<P>(g, d) <= limit && smem_adj<P>(g, d) <= limit && rot_smem_min(d) <= limit &&
            (size_t)d.marea * 4 < (1u << 20))
            return d.nT;
    }
    return 0;
}

template <int P>
cudaError_t fwd_launch(const spect_plan_s& Pl, const float* /*xt: the blur reads the work slab*/, int l0, int nv,
                       cudaStream_t st)
{
    const FusedDims d = dims_for<P>(Pl.g, Pl.fused_J, Pl.fused_nT);
    const size_t smem = smem_fwd<P>(Pl.g, d);
    auto kern = d.nT > 1 ? k_fwd_sep_fused<P, true> : k_fwd_sep_fused<P, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(d.G, nv, d.nT), kFusedThreads, smem, st>>>(Pl.g, d, Pl.slab, Pl.fx, Pl.fz, Pl.part, l0, Pl.err);
    return cudaGetLastError();
}

template <int P>
cudaError_t rot_launch(const spect_plan_s& Pl, const float* xt, int l0, int nv, cudaStream_t st)
{
    const FusedDims d = dims_for<P>(Pl.g, Pl.fused_J, Pl.fused_nT);
    // the three-pass rotation: eight taps per output from its own table
    const size_t smin = Pl.rot3 ? ((size_t)d.farea + (size_t)rot3_ts8(Pl.g.nx)) * sizeof(float) : rot_smem_min(d);
    const size_t smem_mu = smin + (size_t)d.ps * sizeof(float) + 16;
    const bool mus = smem_mu <= (size_t)Pl.smem_optin;
    const size_t smem = mus ? smem_mu : smin;
    auto kern = Pl.rot3 ? (mus ? k_rot_fwd8<P, true> : k_rot_fwd8<P, false>)
                        : (mus ? k_rot_fwd<P, true> : k_rot_fwd<P, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(Pl.g.ny, nv), kRotThreads, smem, st>>>(Pl.g, d, Pl.rot3 ? Pl.r3_tab : Pl.rtab, xt, mubar_for(Pl, l0),
                                                       Pl.slab, l0, Pl.err);
    return cudaGetLastError();
}

template <int P>
cudaError_t adj_launch(const spect_plan_s& Pl, const float* v, int l0, int nv, cudaStream_t st)
{
    const FusedDims d = dims_for<P>(Pl.g, Pl.adj_J, Pl.fused_nT);
    const size_t smem = smem_adj<P>(Pl.g, d);
    auto kern = d.nT > 1 ? k_adj_sep_fused<P, true> : k_adj_sep_fused<P, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(d.G, nv, d.nT), kFusedThreads, smem, st>>>(Pl.g, d, Pl.cls_z, v, mubar_for(Pl, l0), Pl.fx_adj, Pl.fz_adj,
                                                           Pl.slab, l0, Pl.err);
    return cudaGetLastError();
}
}  // namespace

namespace {
template <int P>
size_t dir_smem_fwd(const Geometry& g, const FusedDims& d)
{
    return dir_fwd_smem_floats(d, g.nz, P, Sep<P>::PT, Sep<P>::ZH) * sizeof(float);
}

template <int P>
size_t dir_smem_adj(const Geometry& g, const FusedDims& d, int cls_z)
{
    return dir_adj_smem_floats(d, g.nz, P, Sep<P>::PT, Sep<P>::ZH, 3 * cls_z) * sizeof(float);
}

template <int P>
bool dir_fits(const Geometry& g, size_t limit, int J, int adj_J)
{
    const int cls_z = g.nz >= 2 ? 3 : 1;
    const FusedDims df = dims_for<P>(g, J, 1), da = dims_for<P>(g, adj_J, 1);
    return df.nT == 1 && dir_smem_fwd<P>(g, df) <= limit && dir_smem_adj<P>(g, da, cls_z) <= limit &&
           rot_smem_min(df) <= limit && (size_t)df.ps * 4 < (1u << 20);
}

template <int P>
cudaError_t dir_fwd_launch(const spect_plan_s& Pl, int l0, int nv, cudaStream_t st)
{
    const FusedDims d = dims_for<P>(Pl.g, Pl.fused_J, 1);
    const size_t smem = dir_smem_fwd<P>(Pl.g, d);
    cudaError_t e = cudaFuncSetAttribute(k_fwd_dir_fused<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fwd_dir_fused<P><<<dim3(d.G, nv), kFusedThreads, smem, st>>>(Pl.g, d, Pl.slab, Pl.psf, Pl.part, l0, Pl.err);
    return cudaGetLastError();
}

template <int P>
cudaError_t dir_adj_launch(const spect_plan_s& Pl, const float* v, int l0, int nv, cudaStream_t st)
{
    const FusedDims d = dims_for<P>(Pl.g, Pl.adj_J, 1);
    const size_t smem = dir_smem_adj<P>(Pl.g, d, Pl.cls_z);
    cudaError_t e = cudaFuncSetAttribute(k_adj_dir_fused<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_adj_dir_fused<P><<<dim3(d.G, nv), kFusedThreads, smem, st>>>(Pl.g, d, Pl.cls_z, v, mubar_for(Pl, l0), Pl.psf_adj,
                                                                    Pl.slab, l0, Pl.err);
    return cudaGetLastError();
}
}  // namespace

// Bucket of the fused full-PSF kernels (untiled planes only), 0 when they do not fit.
int fused_dir_bucket(const Geometry& g, size_t smem_limit)
{
    const int p = g.px > g.pz ? g.px : g.pz;
    for (int b : kBuckets) {
        if (b < p) continue;
        bool ok = false;
        switch (b) {
#define SPECT_DF(B) \
    case B: ok = dir_fits<B>(g, smem_limit, 8, 8); break;
            SPECT_DF(3) SPECT_DF(5) SPECT_DF(7) SPECT_DF(9) SPECT_DF(11) SPECT_DF(13) SPECT_DF(15)
            SPECT_DF(17) SPECT_DF(21) SPECT_DF(25) SPECT_DF(29) SPECT_DF(33) SPECT_DF(37)
#undef SPECT_DF
            default: break;
        }
        return ok ? b : 0;
    }
    return 0;
}

int fused_bucket(const Geometry& g, size_t smem_limit, int* tiles)
{
    const int p = g.px > g.pz ? g.px : g.pz;
    *tiles = 0;
    // SPECT_FUSED_TILES: at least this many column tiles (testing and tuning;
    // results are bitwise those of the untiled kernels)
    const char* env = getenv("SPECT_FUSED_TILES");
    const int min_tiles = env ? atoi(env) : 1;
    for (int b : kBuckets) {
        if (b < p) continue;
        int nt = 0;
        switch (b) {
#define SPECT_FITS(B) \
    case B: nt = tiles_that_fit<B>(g, smem_limit, min_tiles); break;
            SPECT_FITS(3) SPECT_FITS(5) SPECT_FITS(7) SPECT_FITS(9) SPECT_FITS(11) SPECT_FITS(13) SPECT_FITS(15)
            SPECT_FITS(17) SPECT_FITS(21) SPECT_FITS(25) SPECT_FITS(29) SPECT_FITS(33) SPECT_FITS(37)
#undef SPECT_FITS
            default: break;
        }
        *tiles = nt;
        return nt > 0 ? b : 0;
    }
    return 0;
}

// Column-tile count the fused kernels use when asked for `tiles` tiles with
// depth groups of J (forward) and adj_J (adjoint) planes, or 0 when that
// configuration does not fit `smem_limit` bytes of shared memory.
int fused_tiles_fit(const Geometry& g, int bucket, int J, int adj_J, int tiles, size_t smem_limit)
{
    auto check = [&](auto tag) -> int {
        constexpr int B = decltype(tag)::value;
        const FusedDims df = dims_for<B>(g, J, tiles), da = dims_for<B>(g, adj_J, tiles);
        const bool ok = smem_fwd<B>(g, df) <= smem_limit && smem_adj<B>(g, da) <= smem_limit &&
                        rot_smem_min(df) <= smem_limit && (size_t)df.marea * 4 < (1u << 20);
        return ok ? df.nT : 0;
    };
    switch (bucket) {
#define SPECT_TF(B) \
    case B: return check(std::integral_constant<int, B>());
        SPECT_TF(3) SPECT_TF(5) SPECT_TF(7) SPECT_TF(9) SPECT_TF(11) SPECT_TF(13) SPECT_TF(15)
        SPECT_TF(17) SPECT_TF(21) SPECT_TF(25) SPECT_TF(29) SPECT_TF(33) SPECT_TF(37)
#undef SPECT_TF
        default: return 0;
    }
}

// Whether the fused full-PSF kernels fit with depth groups J / adj_J.
bool fused_dir_fit(const Geometry& g, int bucket, int J, int adj_J, size_t smem_limit)
{
    switch (bucket) {
#define SPECT_DF(B) \
    case B: return dir_fits<B>(g, smem_limit, J, adj_J);
        SPECT_DF(3) SPECT_DF(5) SPECT_DF(7) SPECT_DF(9) SPECT_DF(11) SPECT_DF(13) SPECT_DF(15)
        SPECT_DF(17) SPECT_DF(21) SPECT_DF(25) SPECT_DF(29) SPECT_DF(33) SPECT_DF(37)
#undef SPECT_DF
        default: return false;
    }
}

int fused_groups(const spect_plan_s& P) { return (P.g.ny + P.fused_J - 1) / P.fused_J; }

#define SPECT_DISPATCH(FN, ...)                        \
    switch (P.bucket) {                                \
        case 3: return FN<3>(__VA_ARGS__);             \
        case 5: return FN<5>(__VA_ARGS__);             \
        case 7: return FN<7>(__VA_ARGS__);             \
        case 9: return FN<9>(__VA_ARGS__);             \
        case 11: return FN<11>(__VA_ARGS__);           \
        case 13: return FN<13>(__VA_ARGS__);           \
        case 15: return FN<15>(__VA_ARGS__);           \
        case 17: return FN<17>(__VA_ARGS__);           \
        case 21: return FN<21>(__VA_ARGS__);           \
        case 25: return FN<25>(__VA_ARGS__);           \
        case 29: return FN<29>(__VA_ARGS__);           \
        case 33: return FN<33>(__VA_ARGS__);           \
        case 37: return FN<37>(__VA_ARGS__);           \
        default: return cudaErrorInvalidValue;         \
    }

cudaError_t launch_fused_forward(const spect_plan_s& P, const float* xt, int l0, int nv, cudaStream_t st)
{
    if (!P.separable) {
        SPECT_DISPATCH(dir_fwd_launch, P, l0, nv, st)
    }
    SPECT_DISPATCH(fwd_launch, P, xt, l0, nv, st)
}

cudaError_t launch_fused_rotate(const spect_plan_s& P, const float* xt, int l0, int nv, cudaStream_t st)
{
    // untiled planes read from the plan's own x_t: the patch-staged rotation (rotpatch.cu)
    if (P.rotpatch && P.rotpatch_on && P.fused_nT == 1 && xt == P.xt) return launch_rot_patch(P, l0, nv, st);
    SPECT_DISPATCH(rot_launch, P, xt, l0, nv, st)
}

namespace {
template <int P>
size_t plane_area(const spect_plan_s& Pl)
{
    return (size_t)dims_for<P>(Pl.g, Pl.fused_J, Pl.fused_nT).parea;
}
}  // namespace

// floats per view of the work slab the fused path needs (rotated tile images or t planes)
size_t fused_slab_per_view(const spect_plan_s& P)
{
    size_t parea = 0;
    switch (P.bucket) {
#define SPECT_AREA(B) \
    case B: parea = plane_area<B>(P); break;
        SPECT_AREA(3) SPECT_AREA(5) SPECT_AREA(7) SPECT_AREA(9) SPECT_AREA(11) SPECT_AREA(13) SPECT_AREA(15)
        SPECT_AREA(17) SPECT_AREA(21) SPECT_AREA(25) SPECT_AREA(29) SPECT_AREA(33) SPECT_AREA(37)
#undef SPECT_AREA
        default: break;
    }
    const size_t ps = ((size_t)P.g.nx * P.g.nz + 3) & ~(size_t)3;
    return (size_t)P.g.ny * (parea > ps ? parea : ps);
}

cudaError_t launch_fused_adjoint(const spect_plan_s& P, const float* v, int l0, int nv, cudaStream_t st)
{
    if (!P.separable) {
        SPECT_DISPATCH(dir_adj_launch, P, v, l0, nv, st)
    }
    SPECT_DISPATCH(adj_launch, P, v, l0, nv, st)
}
#undef SPECT_DISPATCH

cudaError_t launch_fwd_reduce(const spect_plan_s& P, float* v, const float* em_y, const float* em_rbar,
                              cudaStream_t st)
{
    const size_t nproj = (size_t)P.g.nx * P.g.nz * P.g.nview;
    k_fwd_reduce<<<(unsigned)((nproj + 255) / 256), 256, 0, st>>>(P.part, fused_groups(P), nproj, v, em_y, em_rbar);
    return cudaGetLastError();
}

cudaError_t launch_adj_rot_t(const spect_plan_s& P, int l0, int nv, float* out, int accumulate, EmArgs em,
                             cudaStream_t st)
{
    const bool vec4 = (P.g.nz % 4) == 0;
    const size_t n = (size_t)P.g.nx * P.g.ny * (vec4 ? P.g.nz / 4 : P.g.nz);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const float* src = P.slab;
    switch (P.adj_max) {
#define SPECT_ADJ(M)                                                                                                 \
    case M:                                                                                                          \
        if (vec4)                                                                                                    \
            k_adj_rot_t<M, 4><<<blocks, 256, 0, st>>>(P.g, P.ps, P.adjf, src, l0, nv, out, accumulate, em);    \
        else                                                                                                         \
            k_adj_rot_t<M, 1><<<blocks, 256, 0, st>>>(P.g, P.ps, P.adjf, src, l0, nv, out, accumulate, em);    \
        break;
        SPECT_ADJ(1) SPECT_ADJ(2) SPECT_ADJ(3) SPECT_ADJ(4) SPECT_ADJ(5) SPECT_ADJ(6) SPECT_ADJ(7) SPECT_ADJ(8)
#undef SPECT_ADJ
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace spect
