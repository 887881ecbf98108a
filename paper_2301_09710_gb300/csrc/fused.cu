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
#include <cstdlib>
#include <type_traits>

#include "spect_internal.cuh"

namespace spect {

namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Rotation table entry of rotated-frame pixel (i, j): base voxel index
// (i0c + nx*j0c, clamped so all four reads are in bounds) and the four weights
// of slots (0,0), (1,0), (0,1), (1,1) relative to it; neighbours outside the
// slice (zero padding) get weight 0.
__device__ __forceinline__ void rot_table_entry(int i, int j, const ViewRot r, const Geometry& g, float4& w, int& base)
{
    const Sample s = rot_sample(i, j, r, g.cint, g.cfrac);
    const int bi = clampi(s.i0, 0, g.nx - 2), bj = clampi(s.j0, 0, g.ny - 2);
    float ww[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int di = 0; di < 2; ++di) {
            const int qi = s.i0 + di, qj = s.j0 + dj;
            if (qi >= 0 && qi < g.nx && qj >= 0 && qj < g.ny) ww[(qi - bi) + 2 * (qj - bj)] = bilinear_w(s, di, dj);
        }
    w = make_float4(ww[0], ww[1], ww[2], ww[3]);
    base = bi + g.nx * bj;
}

}  // namespace

// ============================================================================
// Plan-time kernels
// ============================================================================

// out[c][r] = in[r][c] for an R x C matrix (tiled through shared memory).
__global__ void k_transpose(const float* __restrict__ in, float* __restrict__ out, int R, int C)
{
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[dy][threadIdx.x] = in[(size_t)r * C + c];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int c = c0 + dy, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * R + r] = tile[threadIdx.x][dy];
    }
}

cudaError_t launch_transpose(const float* in, float* out, int R, int C, cudaStream_t st)
{
    dim3 grid((C + 31) / 32, (R + 31) / 32);
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, out, R, C);
    return cudaGetLastError();
}

// mubar[l][j][i][k] = exp(-dy (mu~(j)/2 + sum_{s>j} mu~(s))), Eq. (1), for every
// view; one thread per (l, i, k) walking j from the detector side.  mu_t is mu
// in the [j][i][k] layout; planes (l, j) are ps floats apart (16-byte aligned
// for bulk copies).
__global__ void k_mubar_cache(Geometry g, int ps, const ViewRot* __restrict__ rot, const float* __restrict__ mu_t,
                              float* __restrict__ mubar)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t per_view = (size_t)g.nx * g.nz;
    if (idx >= per_view * g.nview) return;
    const int l = (int)(idx / per_view);
    const int rem = (int)(idx - (size_t)l * per_view);
    const int i = rem / g.nz, k = rem - i * g.nz;
    const ViewRot r = rot[l];
    AttenScan sc;
    for (int j = g.ny - 1; j >= 0; --j) {
        float4 w;
        int base;
        rot_table_entry(i, j, r, g, w, base);
        const float* m = mu_t + (size_t)base * g.nz + k;
        const size_t rs = (size_t)g.nx * g.nz;
        float mv = 0.f;
        mv = __fmaf_rn(w.x, m[0], mv);
        mv = __fmaf_rn(w.y, m[g.nz], mv);
        mv = __fmaf_rn(w.z, m[rs], mv);
        mv = __fmaf_rn(w.w, m[rs + g.nz], mv);
        mubar[((size_t)l * g.ny + j) * ps + (size_t)i * g.nz + k] = g.has_mu ? sc.step(mv, g.dy) : 1.f;
    }
}

cudaError_t launch_mubar_cache(const spect_plan_s& P, const float* mu_t, cudaStream_t st)
{
    const size_t n = (size_t)P.g.nx * P.g.nz * P.g.nview;
    k_mubar_cache<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P.g, P.ps, P.rot, mu_t, P.mubar);
    return cudaGetLastError();
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

// ============================================================================
// Fused forward, separable PSF, padded tap count P (odd).
//
// The forward runs as two kernels: k_rot_fwd rotates and attenuates every
// (view, depth) plane into the work slab, already in the blur kernel's
// shared-memory image; k_fwd_sep_fused (one block per view and depth group)
// streams those images in by TMA and blurs them.  Its shared memory:
//   W   two plane buffers, nz rows x wp columns: W[k][C + i] with replicate
//       halo columns; wp is a multiple of 4 with wp/4 odd, so the i-pass
//       windows (lanes over k) load as bank-conflict-free float4s.
//   U   nx rows x kpu: i-pass output, U[i][ZH + k], with zero halo columns;
//       kpu/4 is odd so the k-pass float4 windows (lanes over i) are
//       bank-conflict free.  Replicate padding along k enters as folded edge
//       taps: output k adds U(0) sum_{b>k+C} fz(b) + U(nz-1) sum_{b<k+C-nz+1} fz(b).
//   taps and folded edge taps of every plane of the group, staged once.
//   ACC nx x apc depth-sum accumulators of the group, [i][k] (apc/4 odd, so
//       the k-pass float4 read-modify-writes are bank-conflict free).
// Per plane there are two block barriers: after the i-pass (which also agrees
// on the bounded TMA wait) and after the k-pass.
// ============================================================================
template <int P>
struct Sep {
    static constexpr int C = (P - 1) / 2;    // tap centre
    static constexpr int CX = 16;            // i outputs per thread (i-pass)
    static constexpr int CZ = 16;            // k outputs per thread (k-pass)
    static constexpr int ZH = (C + 3) & ~3;  // k halo columns, 16-byte aligned
    static constexpr int WZ = CZ + 2 * ZH;   // k-pass window (multiple of 4)
    static constexpr int PT = (P + 3) & ~3;  // tap array length
};

constexpr int kFusedThreads = 640;

// Shared-memory plan of a fused kernel, computed identically on host and device.
// Planes wider than shared memory allows are cut into nT column tiles of TI
// detector columns (TI a multiple of CX); a tile carries C halo columns on
// each side, so every tile is blurred independently.  nT = 1 is the untiled
// case (TI = nib*CX >= nx).
struct FusedDims {
    int wp;     // W row pitch of one tile image (pitch4odd(TI + 2*C))
    int warea;  // floats of one tile image, nz x wp (multiple of 4, keeps U 16-byte aligned)
    int parea;  // floats of one plane's tile images in the slab, nT x warea
    int kpu;    // U row pitch (>= nkb*CZ + 2*ZH, multiple of 4, pitch/4 odd)
    int nib, nkb;
    int TI, nT; // tile width in columns (multiple of CX), tiles per plane
    int wpf;    // row pitch of the untiled plane image (pitch4odd(nib*CX + 2*C))
    int wz;     // row pitch of the adjoint's Zb (multiple of 4, wz/4 odd: conflict-free float4 windows)
    int zarea;  // floats of Zb, nz x wz
    int farea;  // floats of the untiled plane image (the rotation kernel's shared memory)
    int urows;  // rows of U / ACC / MB per tile: min(TI, nx)
    int vrows;  // detector rows a tile's k-adjoint needs: min(nx, TI + 2*C)
    int marea;  // floats of an attenuation tile, urows*nz rounded up to 4
    int J, G;   // depth planes per block, depth groups
    int ps;     // plane stride of the attenuation cache / slab (nx*nz rounded up to 4)
    int ts;     // rotation table block per (view, row): 5*nx rounded up to 4
    int apc;    // accumulator row pitch (>= nkb*CZ, multiple of 4, pitch/4 odd)
};

__host__ __device__ inline size_t fwd_smem_floats(const FusedDims& d, int nz, int PT)
{
    // W x2 | U | taps J x (FX,FZ) | ACC | folded edge taps J x 2 x (nkb*16) | 2 mbarriers
    (void)nz;
    return 2 * (size_t)d.warea + (size_t)d.urows * d.kpu + 2 * (size_t)PT * d.J + (size_t)d.urows * d.apc +
           2 * (size_t)d.J * d.nkb * 16 + 8;
}

__host__ __device__ inline size_t adj_smem_floats(const FusedDims& d, int PT)
{
    // Zb | V | MB x2 | taps J x (FX[3],FZ[3]) | 2 mbarriers
    return (size_t)d.zarea + (size_t)d.vrows * d.kpu + 2 * (size_t)d.marea + 6 * (size_t)PT * d.J + 8;
}

template <int P>
__device__ __forceinline__ void load_window_f4(const float* base, float (&win)[Sep<P>::WZ])
{
    const float4* row = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int m4 = 0; m4 < Sep<P>::WZ / 4; ++m4) {
        const float4 t = row[m4];
        win[4 * m4] = t.x;
        win[4 * m4 + 1] = t.y;
        win[4 * m4 + 2] = t.z;
        win[4 * m4 + 3] = t.w;
    }
}

// A sliding window along a plane-image row (16-byte aligned, pitch4odd pitch):
// N floats (a multiple of 4) as float4 loads; the FIRs read its first CX + P - 1.
template <int N>
__device__ __forceinline__ void load_row_f4(const float* row, float (&win)[N])
{
    static_assert(N % 4 == 0, "window length must be a multiple of 4");
#pragma unroll
    for (int m4 = 0; m4 < N / 4; ++m4) {
        const float4 t = reinterpret_cast<const float4*>(row)[m4];
        win[4 * m4] = t.x;
        win[4 * m4 + 1] = t.y;
        win[4 * m4 + 2] = t.z;
        win[4 * m4 + 3] = t.w;
    }
}

// o[c] = sum_b taps[b] win[c + SIGN*b + OFF]   (SIGN = -1: convolution, +1: correlation)
template <int P, int N, int SIGN, int OFF, int WN>
__device__ __forceinline__ void fir(const float* taps, const float (&win)[WN], float (&o)[N])
{
    constexpr int PT = Sep<P>::PT;
#pragma unroll
    for (int c = 0; c < N; ++c) o[c] = 0.f;
#pragma unroll
    for (int b4 = 0; b4 < PT / 4; ++b4) {
        const float4 f4 = reinterpret_cast<const float4*>(taps)[b4];
        const float fv[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = 4 * b4 + u;
            if (b < P) {
#pragma unroll
                for (int c = 0; c < N; ++c) o[c] = fmaf(fv[u], win[c + SIGN * b + OFF], o[c]);
            }
        }
    }
}

// sum_b taps[b] w[b + SH] for b = 0..P-1, in that order (one FMA chain)
template <int P, int SH, int N>
__device__ __forceinline__ float tap_dot(const float* taps, const float (&w)[N])
{
    constexpr int PT = Sep<P>::PT;
    static_assert(P - 1 + SH < N, "window too short");
    float s = 0.f;
#pragma unroll
    for (int b4 = 0; b4 < PT / 4; ++b4) {
        const float4 f4 = reinterpret_cast<const float4*>(taps)[b4];
        const float fv[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (4 * b4 + u < P) s = fmaf(fv[u], w[4 * b4 + u + SH], s);
    }
    return s;
}

// sum_b taps[b] row[s + b] for b = 0..P-1 (the edge-class output of an adjoint
// FIR): the samples come in as float4 loads from the aligned position s & ~3
// (row 16-byte aligned, pitch4odd pitch: conflict-free with lanes over rows)
// and the shift s & 3 selects a compile-time offset, so no lane issues P
// dependent scalar loads.  The loads may read up to 3 floats past row[s + P - 1]
// (still inside the caller's shared memory); those are never used.
template <int P>
__device__ __forceinline__ float edge_tap_dot(const float* taps, const float* row, int s)
{
    float w[4 * ((P + 3 + 3) / 4)];
    load_row_f4(row + (s & ~3), w);
    switch (s & 3) {
        case 0: return tap_dot<P, 0>(taps, w);
        case 1: return tap_dot<P, 1>(taps, w);
        case 2: return tap_dot<P, 2>(taps, w);
        default: return tap_dot<P, 3>(taps, w);
    }
}

// Record a timed-out bounded wait in the plan's error word.
__device__ __forceinline__ void flag_timeout(int* err)
{
    if (err) atomicExch(err, (int)SPECT_ETIMEOUT);
}

// ----------------------------------------------------------------------------
// Forward rotation: one block per (depth plane j, view).  Warps take pairs of
// rows i with lanes over k, so the table entry and the four corner pointers
// are warp-uniform and every gather is a coalesced run along k (96 k per
// pass, 30 independent loads per lane in flight).  The plane is
// assembled in shared memory as the blur kernel wants it -- W[k][C+i] with
// replicate halo columns and pitch4odd pitch -- and leaves with one TMA bulk store,
// so the blur kernel can bring it back with one bulk load.  A plane cut into
// column tiles leaves instead as nT tile images W_t[k][c] = W[k][t*TI + c],
// c < TI + 2C, written with coalesced stores.
// ----------------------------------------------------------------------------

constexpr int kRotThreads = 512;

// MUS: the plane's attenuation factors arrive by one TMA bulk load into shared
// memory (issued first, waited for after the first gathers are in flight)
// instead of as per-element global loads, when the two planes fit.
template <int P, bool MUS>
__global__ void __launch_bounds__(kRotThreads, 2) k_rot_fwd(Geometry g, FusedDims d, const float* __restrict__ rtab,
                                                         const float* __restrict__ xt,
                                                         const float* __restrict__ mubar, float* __restrict__ wsl,
                                                         int l0, int* err)
{
    constexpr int C = Sep<P>::C;
    extern __shared__ __align__(16) float sm[];
    float* S = sm;
    float* TBL = sm + d.farea;  // the (view, row) rotation table: nx float4 weights, then nx bases
    float* MU = TBL + d.ts;     // [i][k] attenuation plane (MUS)
    uint64_t* bar = reinterpret_cast<uint64_t*>(MU + d.ps);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = kRotThreads / 32;
    const int j = blockIdx.x, v = blockIdx.y, l = l0 + v;
    const int pln = nx * nz;
    const int wp = d.wpf;
    const int wcols = d.nib * Sep<P>::CX + 2 * C;
    const float* tab = rtab + ((size_t)l * ny + j) * d.ts;
    const float* mb = mubar + ((size_t)l * ny + j) * d.ps;
    if (MUS && threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_load_1d(MU, mb, (unsigned)d.ps * 4u, bar);
    }
    // the table is staged once, so no row step waits on a table load before its gathers
    for (int e = threadIdx.x; e < d.ts / 4; e += kRotThreads)
        reinterpret_cast<float4*>(TBL)[e] = __ldg(reinterpret_cast<const float4*>(tab) + e);
    __syncthreads();  // table staged; the barrier is initialised before anyone waits on it
    const float4* TW = reinterpret_cast<const float4*>(TBL);
    const int* TB = reinterpret_cast<const int*>(TBL + 4 * nx);
    bool ok = true, waited = !MUS;

    for (int i = 2 * warp; i < nx; i += 2 * NW) {
        const bool two = i + 1 < nx;
        const float4 wa = TW[i];
        const float4 wb = two ? TW[i + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float* pa = xt + (size_t)TB[i] * nz;
        const float* pb = xt + (size_t)TB[two ? i + 1 : i] * nz;
        for (int k0 = 0; k0 < nz; k0 += 96) {
            float xa[3][4], xb[3][4], ma[3], mc[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int k = k0 + 32 * q + lane;
                if (k < nz) {
                    xa[q][0] = __ldg(pa + k);
                    xa[q][1] = __ldg(pa + nz + k);
                    xa[q][2] = __ldg(pa + pln + k);
                    xa[q][3] = __ldg(pa + pln + nz + k);
                    xb[q][0] = __ldg(pb + k);
                    xb[q][1] = __ldg(pb + nz + k);
                    xb[q][2] = __ldg(pb + pln + k);
                    xb[q][3] = __ldg(pb + pln + nz + k);
                    if (!MUS) {
                        ma[q] = __ldg(mb + i * nz + k);
                        mc[q] = two ? __ldg(mb + (i + 1) * nz + k) : 0.f;
                    }
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
                    if (MUS) {
                        ma[q] = MU[i * nz + k];
                        mc[q] = two ? MU[(i + 1) * nz + k] : 0.f;
                    }
                    float* wr = S + k * wp + C;
                    float va = wa.x * xa[q][0];
                    va = fmaf(wa.y, xa[q][1], va);
                    va = fmaf(wa.z, xa[q][2], va);
                    va = fmaf(wa.w, xa[q][3], va);
                    va *= ma[q];
                    if (two) {
                        float vb = wb.x * xb[q][0];
                        vb = fmaf(wb.y, xb[q][1], vb);
                        vb = fmaf(wb.z, xb[q][2], vb);
                        vb = fmaf(wb.w, xb[q][3], vb);
                        vb *= mc[q];
                        if (C % 2 == 0) {  // i even: one 8-byte store (half the bank conflicts of two)
                            *reinterpret_cast<float2*>(wr + i) = make_float2(va, vb);
                        } else {
                            wr[i] = va;
                            wr[i + 1] = vb;
                        }
                        if (i + 1 == nx - 1)
                            for (int h = nx; h < wcols - C; ++h) wr[h] = vb;
                    } else {
                        wr[i] = va;
                    }
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
    // tile images: row k of tile t is W[k][t*TI .. t*TI + TI + 2C), cut at
    // the end of the plane's row (the blur never reads past it)
    for (int r = warp; r < d.nT * nz; r += NW) {
        const int t = r / nz, k = r - t * nz;
        const int tw = min(d.TI + 2 * C, wcols - t * d.TI);
        const float* src = S + k * wp + t * d.TI;
        float* out = dst + (size_t)t * d.warea + (size_t)k * d.wp;
        for (int c = lane; c < tw; c += 32) out[c] = src[c];
    }
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
    using S = Sep<P>;
    constexpr int C = S::C, CX = S::CX, CZ = S::CZ, ZH = S::ZH, WZ = S::WZ, PT = S::PT;
    extern __shared__ __align__(16) float sm[];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    float* WB = sm;                                    // [2][warea]
    float* U = WB + 2 * (size_t)d.warea;
    float* TAP = U + (size_t)d.urows * d.kpu;          // [J][FX PT | FZ PT], every plane of the group
    float* ACC = TAP + 2 * PT * (size_t)d.J;           // urows x apc, [i - i0][k]
    const int fs = d.nkb * CZ;                          // folded-tap row length (zero beyond nz)
    float* FOLD = ACC + (size_t)d.urows * d.apc;        // [J][2][fs] folded edge taps of the k-pass
    uint64_t* bar = reinterpret_cast<uint64_t*>(FOLD + 2 * (size_t)d.J * fs);
    const int tid = threadIdx.x;
    constexpr int T = kFusedThreads;
    const int grp = blockIdx.x, v = blockIdx.y, l = l0 + v;
    // this tile's columns (untiled: the whole plane, constants folded at compile time)
    const int i0 = TILED ? (int)blockIdx.z * d.TI : 0;
    const int ti = TILED ? min(d.TI, nx - i0) : nx;
    const int nibt = TILED ? (ti + CX - 1) / CX : d.nib;
    const int lp = g.nvp == 1 ? 0 : l;
    const int j_begin = grp * d.J, j_end = min(ny, j_begin + d.J);
    const int ox = (P - g.px) / 2, oz = (P - g.pz) / 2;  // zero-padding offsets of the taps
    const int pln = nx * nz;
    // tile blockIdx.z of plane j sits at wv + j * parea
    const float* wv = wsl + (size_t)v * ny * d.parea + (size_t)blockIdx.z * d.warea;

    // taps of every plane of the group (zero-padded to P, centred)
    for (int e = tid; e < (j_end - j_begin) * PT; e += T) {
        const int jj = e / PT, a = e - jj * PT, j = j_begin + jj;
        const int ax = a - ox, az = a - oz;
        TAP[jj * 2 * PT + a] = (ax >= 0 && ax < g.px) ? __ldg(fx + ((size_t)lp * ny + j) * g.px + ax) : 0.f;
        TAP[jj * 2 * PT + PT + a] = (az >= 0 && az < g.pz) ? __ldg(fz + ((size_t)lp * ny + j) * g.pz + az) : 0.f;
    }
    for (int e = tid; e < d.urows * d.apc; e += T) ACC[e] = 0.f;
    for (int e = tid; e < d.urows * d.kpu; e += T) U[e] = 0.f;  // zero k-halo columns (never written again)
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_load_1d(WB, wv + (size_t)j_begin * d.parea, (unsigned)d.warea * 4u, bar);
        if (j_begin + 1 < j_end)
            tma_load_1d(WB + d.warea, wv + (size_t)(j_begin + 1) * d.parea, (unsigned)d.warea * 4u, bar + 1);
    }
    __syncthreads();
    // replicate padding along k, folded: output k takes U(0) * sum_{b > k+C} fz(b)
    // and U(nz-1) * sum_{b < k+C-nz+1} fz(b) on top of the zero-padded k-pass
    for (int e = tid; e < (j_end - j_begin) * fs; e += T) {
        const int jj = e / fs, k = e - jj * fs;
        const float* f = TAP + jj * 2 * PT + PT;
        float lo = 0.f, hi = 0.f;
        if (k < nz) {
            for (int bq = k + C + 1; bq < P; ++bq) lo += f[bq];
            for (int bq = 0; bq < k + C - nz + 1 && bq < P; ++bq) hi += f[bq];
        }
        FOLD[(jj * 2) * fs + k] = lo;
        FOLD[(jj * 2 + 1) * fs + k] = hi;
    }
    __syncthreads();

    // the thread's first work item of each pass and the step to its next one
    // (the same for every plane: the divisions stay out of the plane loop)
    const int ip_ib = tid / nz, ip_k = tid - ip_ib * nz;    // i-pass: (column run, k)
    const int kp_kb = tid / ti, kp_i = tid - kp_kb * ti;    // k-pass: (k run, column)
    const int ip_dib = T / nz, ip_dk = T - ip_dib * nz;
    const int kp_dkb = T / ti, kp_di = T - kp_dkb * ti;
    unsigned phases = 0u;                                   // bit b: parity of buffer b's barrier
    for (int j = j_begin; j < j_end; ++j) {
        const int b = (j - j_begin) & 1;
        const float* FX = TAP + (j - j_begin) * 2 * PT;
        const float* FZ = FX + PT;
        const float* W = WB + b * (size_t)d.warea;
        const bool ok = mbar_wait_bounded(bar + b, (phases >> b) & 1u);
        phases ^= 1u << b;

        // i-pass: U(i,k) = sum_a fx(a) w(clamp(i-a+cx), k); lanes over k
        if (ok) {
            int ib = ip_ib, k = ip_k;
            for (int it = tid; it < nz * nibt; it += T) {
                const int li = ib * CX;  // first column of this run, relative to the tile
                const float* wr = W + k * d.wp + li;
                float win[4 * ((CX + P - 1 + 3) / 4)];
                load_row_f4(wr, win);
                float o[CX];
                fir<P, CX, -1, P - 1>(FX, win, o);
                float* ur = U + li * d.kpu + ZH + k;
                if (li + CX <= ti) {
#pragma unroll
                    for (int c = 0; c < CX; ++c) ur[c * d.kpu] = o[c];
                } else {
#pragma unroll
                    for (int c = 0; c < CX; ++c)
                        if (li + c < ti) ur[c * d.kpu] = o[c];
                }
                ib += ip_dib;  // next item: it + T
                k += ip_dk;
                if (k >= nz) k -= nz, ++ib;
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                flag_timeout(err);
                mbar_wait_bounded(bar + b, ((phases >> b) & 1u) ^ 1u);  // a last chance for the copies in flight
                mbar_wait_bounded(bar + (b ^ 1), (phases >> (b ^ 1)) & 1u);
            }
            return;
        }
        // buffer b has been read: request plane j+2 into it (from the last warp,
        // which has the fewest halo rows below)
        if (tid == T - 32 && j + 2 < j_end) {
            fence_proxy_async_smem();
            tma_load_1d(WB + b * (size_t)d.warea, wv + (size_t)(j + 2) * d.parea, (unsigned)d.warea * 4u, bar + b);
        }

        // k-pass into the depth-sum accumulators: lanes over i; zero-padded
        // FIR plus the folded replicate-padding terms on the edge rows
        const float* fold_lo = FOLD + (j - j_begin) * 2 * fs;
        const float* fold_hi = fold_lo + fs;
        int kb = kp_kb, i = kp_i;  // i relative to the tile
        for (int it = tid; it < ti * d.nkb; it += T) {
            const float* ur = U + i * d.kpu;
            float win[WZ];
            load_window_f4<P>(ur + kb * CZ, win);
            float o[CZ];
            fir<P, CZ, -1, C + ZH>(FZ, win, o);
            const int k0 = kb * CZ;
            // folded taps are zero outside the first and last C rows
            if (k0 + CZ > nz - C) {
                const float uhi = ur[ZH + nz - 1];
                const float4* f4 = reinterpret_cast<const float4*>(fold_hi + k0);
#pragma unroll
                for (int c4 = 0; c4 < CZ / 4; ++c4) {
                    const float4 f = f4[c4];
                    o[4 * c4] = fmaf(uhi, f.x, o[4 * c4]);
                    o[4 * c4 + 1] = fmaf(uhi, f.y, o[4 * c4 + 1]);
                    o[4 * c4 + 2] = fmaf(uhi, f.z, o[4 * c4 + 2]);
                    o[4 * c4 + 3] = fmaf(uhi, f.w, o[4 * c4 + 3]);
                }
            }
            if (k0 < C) {
                const float ulo = ur[ZH];
                const float4* f4 = reinterpret_cast<const float4*>(fold_lo + k0);
#pragma unroll
                for (int c4 = 0; c4 < CZ / 4; ++c4) {
                    const float4 f = f4[c4];
                    o[4 * c4] = fmaf(ulo, f.x, o[4 * c4]);
                    o[4 * c4 + 1] = fmaf(ulo, f.y, o[4 * c4 + 1]);
                    o[4 * c4 + 2] = fmaf(ulo, f.z, o[4 * c4 + 2]);
                    o[4 * c4 + 3] = fmaf(ulo, f.w, o[4 * c4 + 3]);
                }
            }
            float4* acc4 = reinterpret_cast<float4*>(ACC + i * d.apc + kb * CZ);
#pragma unroll
            for (int c4 = 0; c4 < CZ / 4; ++c4) {
                float4 a = acc4[c4];
                a.x += o[4 * c4];
                a.y += o[4 * c4 + 1];
                a.z += o[4 * c4 + 2];
                a.w += o[4 * c4 + 3];
                acc4[c4] = a;
            }
            kb += kp_dkb;  // next item: it + T
            i += kp_di;
            if (i >= ti) i -= ti, ++kb;
        }
        __syncthreads();
    }

    // partial depth sums of this group: part[grp][l][k][i], this tile's columns
    float* pout = part + ((size_t)grp * g.nview + l) * pln + i0;
    for (int e = tid; e < nz * ti; e += T) {
        const int k = e / ti, i = e - k * ti;
        pout[(size_t)k * nx + i] = ACC[i * d.apc + k];
    }
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

// ============================================================================
// Fused transpose of the blur + attenuation, separable PSF.
//   V   nx rows x kpu: the detector plane, V[i][ZH + k], zero halo columns
//   Zb  nz rows x wp: k-adjoint of every V row, Zb[k][C + i], zero halo columns
//   MB  two plane buffers: each receives mubar(:, j, :) by TMA, is overwritten
//       in place with t = wbar * mubar, and leaves for the slab by a TMA bulk
//       store; the buffer of plane j+1 is loaded while plane j is computed.
// ============================================================================
template <int P, bool TILED>
__global__ void __launch_bounds__(kFusedThreads, 1) k_adj_sep_fused(Geometry g, FusedDims d, int cls_z,
                                                                     const float* __restrict__ vin,
                                                                     const float* __restrict__ mubar,
                                                                     const float* __restrict__ fx_adj,
                                                                     const float* __restrict__ fz_adj,
                                                                     float* __restrict__ slab, int l0, int* err)
{
    using S = Sep<P>;
    constexpr int C = S::C, CX = S::CX, CZ = S::CZ, ZH = S::ZH, WZ = S::WZ, PT = S::PT;
    extern __shared__ __align__(16) float sm[];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    float* Zb = sm;
    float* V = Zb + d.zarea;
    float* MB = V + (size_t)d.vrows * d.kpu;  // [2][marea]
    float* TAP = MB + 2 * (size_t)d.marea;    // [J][FX 3 classes | FZ 3 classes] x PT, every plane of the group
    uint64_t* bar = reinterpret_cast<uint64_t*>(TAP + 6 * PT * (size_t)d.J);
    const int tid = threadIdx.x;
    constexpr int T = kFusedThreads;
    const int grp = blockIdx.x, v = blockIdx.y, l = l0 + v;
    // output columns [i0, i0 + ti); their i-adjoint reads detector rows [vlo, vhi)
    // (untiled: the whole plane, with the constants folded at compile time)
    const int i0 = TILED ? (int)blockIdx.z * d.TI : 0;
    const int ti = TILED ? min(d.TI, nx - i0) : nx;
    const int vlo = TILED ? max(0, i0 - C) : 0;
    const int nvr = TILED ? min(nx, i0 + d.TI + C) - vlo : nx;
    const int nibt = TILED ? (ti + CX - 1) / CX : d.nib;
    const int zoff = C + vlo - i0;       // Zb column of detector row vlo
    const int last_col = nx - 1 - i0;    // tile-relative position of column nx-1
    const bool first_tile = i0 == 0;
    // attenuation / t tile: columns [i0, i0 + ti) of a plane are one contiguous run
#define SPECT_MBYTES ((unsigned)(((size_t)ti * nz + 3) & ~(size_t)3) * 4u)
    const int lp = g.nvp == 1 ? 0 : l;
    const int j_begin = grp * d.J, j_end = min(ny, j_begin + d.J);
    const int ox = (P - g.px) / 2, oz = (P - g.pz) / 2;
    const size_t nrow = (size_t)g.nvp * ny;
    const int pln = nx * nz;
    const float* mub = mubar + ((size_t)l * ny) * d.ps + (size_t)i0 * nz;
    float* tsl = slab + ((size_t)v * ny) * d.ps + (size_t)i0 * nz;

    // edge-class taps of every plane of the group
    for (int e = tid; e < (j_end - j_begin) * 3 * PT; e += T) {
        const int jj = e / (3 * PT), r3 = e - jj * 3 * PT, c = r3 / PT, a = r3 - c * PT, j = j_begin + jj;
        const int ax = a - ox, az = a - oz;
        float* F = TAP + jj * 6 * PT;
        F[r3] = (ax >= 0 && ax < g.px) ? __ldg(fx_adj + ((size_t)c * nrow + (size_t)lp * ny + j) * g.px + ax) : 0.f;
        F[3 * PT + r3] = (c < cls_z && az >= 0 && az < g.pz)
                             ? __ldg(fz_adj + ((size_t)c * nrow + (size_t)lp * ny + j) * g.pz + az)
                             : 0.f;
    }

    // stage the detector plane v(:,:,l) transposed, zero outside the detector
    for (int e = tid; e < d.vrows * d.kpu; e += T) V[e] = 0.f;
    for (int e = tid; e < d.zarea; e += T) Zb[e] = 0.f;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_load_1d(MB, mub + (size_t)j_begin * d.ps, SPECT_MBYTES, bar);
    }
    __syncthreads();
    for (int e = tid; e < nz * nvr; e += T) {
        const int k = e / nvr, r = e - k * nvr;
        V[r * d.kpu + ZH + k] = vin[(size_t)l * pln + (size_t)k * nx + vlo + r];
    }
    __syncthreads();

    // the thread's first work item of each pass and the step to its next one
    // (the same for every plane: the divisions stay out of the plane loop)
    const int ka_kb = tid / nvr, ka_r = tid - ka_kb * nvr;  // k-adjoint: (k run, detector row)
    const int ka_dkb = T / nvr, ka_dr = T - ka_dkb * nvr;
    const int ia_ib = tid / nz, ia_k = tid - ia_ib * nz;    // i-adjoint: (column run, k)
    const int ia_dib = T / nz, ia_dk = T - ia_dib * nz;
    unsigned phases = 0u;  // bit b: parity of buffer b's barrier
    for (int j = j_begin; j < j_end; ++j) {
        const int n = j - j_begin, b = n & 1;
        const float* FX = TAP + n * 6 * PT;
        const float* FZ = FX + 3 * PT;
        // k-adjoint: Zb[k][C+i] = sum_b' fz~(b') v(i, k+b'-cz), lanes over i.
        // The first and last detector rows, where replicate padding folds
        // taps together, take their edge-class taps instead of the interior ones.
        int kb = ka_kb, r = ka_r;  // detector row vlo + r
        for (int it = tid; it < nvr * d.nkb; it += T, kb += ka_dkb, r += ka_dr) {
            if (r >= nvr) r -= nvr, ++kb;
            const float* vr = V + r * d.kpu;
            float win[WZ];
            load_window_f4<P>(vr + kb * CZ, win);
            float o[CZ];
            fir<P, CZ, 1, ZH - C>(FZ, win, o);
            const int k0 = kb * CZ;
            if (nz > 1 && k0 == 0) {  // row k = 0
                const float* f = FZ + PT;
                float sacc = 0.f;
#pragma unroll
                for (int bb = 0; bb < P; ++bb) sacc = fmaf(f[bb], win[bb - C + ZH], sacc);
                o[0] = sacc;
            }
            const int cl = nz - 1 - k0;  // position of row k = nz-1 in this block
            const bool last = nz > 1 && cl < CZ;
            const float e_last = last ? edge_tap_dot<P>(FZ + 2 * PT, vr, (nz - 1) - C + ZH) : 0.f;
            float* zc = Zb + zoff + r;
            if (k0 + CZ <= nz && !last) {
#pragma unroll
                for (int c = 0; c < CZ; ++c) zc[(k0 + c) * d.wz] = o[c];
            } else {
#pragma unroll
                for (int c = 0; c < CZ; ++c)
                    if (k0 + c < nz) zc[(k0 + c) * d.wz] = (last && c == cl) ? e_last : o[c];
            }
        }
        __syncthreads();
        // the other buffer: the previous plane's bulk store has had the whole
        // k-adjoint to read it; it now receives the next plane's attenuation
        if (tid == 0 && j + 1 < j_end) {
            tma_store_wait_read<0>();
            tma_load_1d(MB + (b ^ 1) * (size_t)d.marea, mub + (size_t)(j + 1) * d.ps, SPECT_MBYTES, bar + (b ^ 1));
        }

        // i-adjoint times mubar, in place in MB[b]; lanes over k
        float* mb = MB + b * (size_t)d.marea;
        const bool ok = mbar_wait_bounded(bar + b, (phases >> b) & 1u);
        phases ^= 1u << b;
        if (ok) {
            int ib = ia_ib, k = ia_k;
            for (int it = tid; it < nz * nibt; it += T, ib += ia_dib, k += ia_dk) {
                if (k >= nz) k -= nz, ++ib;
                const int li = ib * CX;  // first column of this run, relative to the tile
                const float* zr = Zb + k * d.wz + li;
                float win[4 * ((CX + P - 1 + 3) / 4)];
                load_row_f4(zr, win);
                float o[CX];
                fir<P, CX, 1, 0>(FX, win, o);
                // first / last detector column: edge-class taps (replicate-padding folds)
                if (first_tile && li == 0) {
                    const float* f = FX + PT;
                    float sacc = 0.f;
#pragma unroll
                    for (int a = 0; a < P; ++a) sacc = fmaf(f[a], win[a], sacc);
                    o[0] = sacc;
                }
                const int cl = last_col - li;  // position of column nx-1 in this run
                const bool last = cl < CX;
                const float e_last = last ? edge_tap_dot<P>(FX + 2 * PT, zr - li, li + cl) : 0.f;
                float* mp = mb + li * nz + k;
                if (!last) {
#pragma unroll
                    for (int c = 0; c < CX; ++c) mp[c * nz] = o[c] * mp[c * nz];
                } else {
#pragma unroll
                    for (int c = 0; c < CX; ++c)
                        if (c <= cl) mp[c * nz] = (c == cl ? e_last : o[c]) * mp[c * nz];
                }
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
        // t plane -> slab[v][j]
        if (tid == 0) {
            fence_proxy_async_smem();
            tma_store_1d(tsl + (size_t)j * d.ps, mb, SPECT_MBYTES);
        }
    }
    if (tid == 0) tma_store_wait_read<0>();  // the writes complete with the grid
#undef SPECT_MBYTES
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
constexpr int kBuckets[] = {3, 5, 7, 9, 11, 13, 15, 17, 21, 25, 29, 33, 37};

template <int P>
FusedDims dims_for(const Geometry& g, int J, int tiles)
{
    using S = Sep<P>;
    FusedDims d;
    d.ps = (g.nx * g.nz + 3) & ~3;
    d.ts = (5 * g.nx + 3) & ~3;
    d.nib = (g.nx + S::CX - 1) / S::CX;
    d.nkb = (g.nz + S::CZ - 1) / S::CZ;
    tiles = tiles < 1 ? 1 : (tiles > d.nib ? d.nib : tiles);
    d.TI = ((d.nib + tiles - 1) / tiles) * S::CX;
    d.nT = (g.nx + d.TI - 1) / d.TI;
    d.urows = d.TI < g.nx ? d.TI : g.nx;
    d.vrows = d.TI + 2 * S::C < g.nx ? d.TI + 2 * S::C : g.nx;
    d.marea = (d.urows * g.nz + 3) & ~3;
    d.wp = pitch4odd(d.TI + 2 * S::C);
    d.warea = (g.nz * d.wp + 3) & ~3;
    d.parea = d.nT * d.warea;
    d.wpf = pitch4odd(d.nib * S::CX + 2 * S::C);
    d.wz = pitch4odd(d.TI + 2 * S::C);
    d.zarea = g.nz * d.wz;
    d.farea = (g.nz * d.wpf + 3) & ~3;
    int kpu = d.nkb * S::CZ + 2 * S::ZH;
    kpu = (kpu + 3) & ~3;
    if (((kpu / 4) & 1) == 0) kpu += 4;
    d.kpu = kpu;
    int apc = d.nkb * S::CZ;
    if (((apc / 4) & 1) == 0) apc += 4;
    d.apc = apc;
    d.J = J;
    d.G = (g.ny + J - 1) / J;
    return d;
}

// Rotation kernel without the attenuation plane staged: plane image + table.
inline size_t rot_smem_min(const FusedDims& d) { return ((size_t)d.farea + d.ts) * sizeof(float); }

template <int P>
size_t smem_fwd(const Geometry& g, const FusedDims& d)
{
    return fwd_smem_floats(d, g.nz, Sep<P>::PT) * sizeof(float);
}

template <int P>
size_t smem_adj(const Geometry& g, const FusedDims& d)
{
    (void)g;
    return adj_smem_floats(d, Sep<P>::PT) * sizeof(float);
}

// The fewest column tiles with which the rotation, blur and adjoint kernels
// fit `limit` bytes of shared memory (and every bulk copy stays below the
// mbarrier's 2^20-byte transaction count); 0 when none does.
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
cudaError_t fwd_launch(const spect_plan_s& Pl, const float* xt, int l0, int nv, cudaStream_t st)
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
    kern<<<dim3(Pl.g.ny, nv), kRotThreads, smem, st>>>(Pl.g, d, Pl.rot3 ? Pl.r3_tab : Pl.rtab, xt, Pl.mubar,
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
    kern<<<dim3(d.G, nv, d.nT), kFusedThreads, smem, st>>>(Pl.g, d, Pl.cls_z, v, Pl.mubar, Pl.fx_adj, Pl.fz_adj,
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
    k_adj_dir_fused<P><<<dim3(d.G, nv), kFusedThreads, smem, st>>>(Pl.g, d, Pl.cls_z, v, Pl.mubar, Pl.psf_adj,
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
