// rotate.cu -- rotation steps of the projector (Section II-A, Algorithms 1-2):
//   K1  rotate x and mu by theta_l, Eq. (1) attenuation, w = x~ * mubar
//   K1T transpose of the bilinear rotation as a gather over destination
//       voxels (owner computes, no atomics), summed over views
//   the plan-time builder of K1T's adjacency lists.
#include "spect_internal.cuh"

namespace spect {

// ----------------------------------------------------------------------------
// K1: w(i,j,k; v) = x~(i,j,k) * mubar(i,j,k), rotation and Eq. (1) attenuation
// fused.  One block per (32 columns i, slice k, view): it walks depth from the
// detector side in tiles of 32 depths; per tile the rotated x~ and mu~ are
// gathered with lanes over i, each warp scans four columns of mu~ along depth
// (atten_warp_scan, lanes over depth) into the factors mubar, and w = x~ mubar
// leaves with lanes over i (coalesced rows of the slab).
// Output: slab[v][k][j][i].
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rotate_atten(Geometry g, const ViewRot* __restrict__ rot,
                                                      const float* __restrict__ x, const float* __restrict__ mu,
                                                      float* __restrict__ slab, int l0)
{
    __shared__ float tx[32][33], tm[32][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane, k = blockIdx.y, v = blockIdx.z;
    const ViewRot r = rot[l0 + v];
    const size_t nxy = (size_t)g.nx * g.ny;
    const float* xs = x + (size_t)k * nxy;
    const float* ms = mu + (size_t)k * nxy;
    float* out = slab + ((size_t)v * g.nz + k) * nxy;
    DFloat carry[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};  // columns warp + 8t
    for (int j0 = g.ny - 1; j0 >= 0; j0 -= 32) {  // depths j0, j0-1, ..., j0-31
        for (int q = warp; q < 32; q += 8) {
            const int j = j0 - q;
            float xv = 0.f, mv = 0.f;
            if (j >= 0 && i < g.nx) {
                const Sample s = rot_sample(i, j, r, g.cint, g.cfrac);
                xv = gather_bilinear(xs, s, g.nx, g.ny);
                if (g.has_mu) mv = gather_bilinear(ms, s, g.nx, g.ny);
            }
            tx[q][lane] = xv;
            tm[q][lane] = mv;
        }
        __syncthreads();
        if (g.has_mu) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int c = warp + 8 * t;
                tx[lane][c] *= atten_warp_scan(tm[lane][c], carry[t], g.dy);
            }
        }
        __syncthreads();
        for (int q = warp; q < 32; q += 8) {
            const int j = j0 - q;
            if (j >= 0 && i < g.nx) out[(size_t)j * g.nx + i] = tx[q][lane];
        }
        __syncthreads();
    }
}

cudaError_t launch_rotate_atten(const spect_plan_s& P, const float* x, int l0, int nv, cudaStream_t st)
{
    const Geometry& g = P.g;
    dim3 grid((g.nx + 31) / 32, g.nz, nv);
    k_rotate_atten<<<grid, 256, 0, st>>>(g, P.rot, x, P.mu, P.slab, l0);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// K1T: out(q,k) (+)= sum_{v in chunk} sum_{(p,w) in adj(l0+v, q)} w * t(p,k; v)
// The adjacency list of destination q holds every rotated-frame pixel p whose
// bilinear stencil covers q, with the same FP32 weight K1 uses.
// With em.x set, the final value e is turned into the EM update of em.x
// (em_update: MLEM, or the regularised form when em.beta > 0) instead of
// being stored.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rotate_adjoint(Geometry g, const int* __restrict__ adj_off,
                                                        const AdjEntry* __restrict__ adj,
                                                        const float* __restrict__ slab, int l0, int nv,
                                                        float* out, int accumulate, EmArgs em)
{
    const size_t nxy = (size_t)g.nx * g.ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nxy * g.nz) return;
    const size_t q = idx % nxy, k = idx / nxy;
    KSum acc;
    for (int v = 0; v < nv; ++v) {
        const float* t = slab + ((size_t)v * g.nz + k) * nxy;
        const size_t row = (size_t)(l0 + v) * nxy + q;
        const int b = __ldg(adj_off + row), e = __ldg(adj_off + row + 1);
        for (int m = b; m < e; ++m) {
            const AdjEntry a = adj[m];
            acc.add(a.w * __ldg(t + a.p));
        }
    }
    const size_t o = k * nxy + q;
    float val = acc.value();
    if (accumulate) val += out[o];
    if (em.x) em.x[o] = em_update(em.x[o], val, em.s[o], em.u ? em.u[o] : 0.f, em.beta);
    else out[o] = val;
}

cudaError_t launch_rotate_adjoint(const spect_plan_s& P, int l0, int nv, float* out, int accumulate, EmArgs em,
                                  cudaStream_t st)
{
    const Geometry& g = P.g;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    k_rotate_adjoint<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, P.adj_off, P.adj, P.slab, l0, nv, out,
                                                                  accumulate, em);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Adjacency builder (plan time).  For destination q = (qi,qj) and view l the
// source pixels p with q in their bilinear stencil satisfy
// |s(p) - q|_inf < 1, hence |p - p*|_inf < |cos| + |sin| <= sqrt(2) with
// p* = c + R(theta)^T (q - c): a 4x4 box of candidates covers them.  Every
// candidate is re-sampled with rot_sample(), the function K1 uses, so the
// weights are bitwise those of A.  pass 0 counts, pass 1 fills (in the fixed
// candidate order, so the lists are deterministic).
// ----------------------------------------------------------------------------
__global__ void k_build_adjacency(Geometry g, const ViewRot* __restrict__ rot, int pass, int* counts,
                                  int* maxcount, const int* __restrict__ off, AdjEntry* adj)
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
    int cnt = 0;
    const int base = pass == 1 ? off[idx] : 0;
    for (int cj = 0; cj < 4; ++cj)
        for (int ci = 0; ci < 4; ++ci) {
            const int pi = bi + ci, pj = bj + cj;
            if (pi < 0 || pi >= g.nx || pj < 0 || pj >= g.ny) continue;
            const Sample s = rot_sample(pi, pj, r, g.cint, g.cfrac);
            const int di = qi - s.i0, dj = qj - s.j0;
            if (di < 0 || di > 1 || dj < 0 || dj > 1) continue;
            const float w = bilinear_w(s, di, dj);
            if (w == 0.f) continue;
            if (pass == 1) {
                AdjEntry e;
                e.p = pi + g.nx * pj;
                e.w = w;
                adj[base + cnt] = e;
            }
            ++cnt;
        }
    if (pass == 0) {
        counts[idx] = cnt;
        atomicMax(maxcount, cnt);
    }
}

cudaError_t launch_build_adjacency(const spect_plan_s& P, int pass, int* counts, int* maxcount, cudaStream_t st)
{
    const Geometry& g = P.g;
    const size_t n = (size_t)g.nx * g.ny * g.nview;
    k_build_adjacency<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, P.rot, pass, counts, maxcount, P.adj_off,
                                                                   P.adj);
    return cudaGetLastError();
}

__global__ void k_fill(float* p, size_t n, float value)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = value;
}

cudaError_t launch_fill(float* p, size_t n, float value, cudaStream_t st)
{
    k_fill<<<1024, 256, 0, st>>>(p, n, value);
    return cudaGetLastError();
}

}  // namespace spect
