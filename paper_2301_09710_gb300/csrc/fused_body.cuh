// fused_body.cuh -- device bodies of the fused projector kernels (rotation,
// separable blur + depth sum, blur adjoint + attenuation), their helpers and
// their host-side dimensioning, shared by the per-plan launches (fused.cu) and
// the grouped launches over many plans (grouped.cu).  The kernels themselves
// are thin wrappers that pass their block coordinates to these bodies, so a
// block computes the same values whichever launch runs it.
#pragma once

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

// out[c][r] = in[r][c] for the 32x32 tile (bx, by) of an R x C matrix (tiled
// through shared memory; blocks of 32 x 8 threads).
__device__ __forceinline__ void transpose_body(const float* __restrict__ in, float* __restrict__ out, int R, int C,
                                               int bx, int by)
{
    __shared__ float tile[32][33];
    const int c0 = bx * 32, r0 = by * 32;
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
__device__ __forceinline__ void rot_fwd_body(const Geometry& g, const FusedDims& d, const float* __restrict__ rtab,
                                             const float* __restrict__ xt, const float* __restrict__ mubar,
                                             float* __restrict__ wsl, int l0, int* err, const int j, const int v)
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
    const int l = l0 + v;
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

template <int P, bool TILED>
__device__ __forceinline__ void fwd_sep_body(const Geometry& g, const FusedDims& d, const float* __restrict__ wsl,
                                             const float* __restrict__ fx, const float* __restrict__ fz,
                                             float* __restrict__ part, int l0, int* err, const int grp, const int v,
                                             const int tile)
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
    const int l = l0 + v;
    // this tile's columns (untiled: the whole plane, constants folded at compile time)
    const int i0 = TILED ? (int)tile * d.TI : 0;
    const int ti = TILED ? min(d.TI, nx - i0) : nx;
    const int nibt = TILED ? (ti + CX - 1) / CX : d.nib;
    const int lp = g.nvp == 1 ? 0 : l;
    const int j_begin = grp * d.J, j_end = min(ny, j_begin + d.J);
    const int ox = (P - g.px) / 2, oz = (P - g.pz) / 2;  // zero-padding offsets of the taps
    const int pln = nx * nz;
    // tile `tile` of plane j sits at wv + j * parea
    const float* wv = wsl + (size_t)v * ny * d.parea + (size_t)tile * d.warea;

    // the first two plane images are requested before anything else, so their
    // loads overlap the set-up below
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_load_1d(WB, wv + (size_t)j_begin * d.parea, (unsigned)d.warea * 4u, bar);
        if (j_begin + 1 < j_end)
            tma_load_1d(WB + d.warea, wv + (size_t)(j_begin + 1) * d.parea, (unsigned)d.warea * 4u, bar + 1);
    }
    // taps of every plane of the group (zero-padded to P, centred)
    for (int e = tid; e < (j_end - j_begin) * PT; e += T) {
        const int jj = e / PT, a = e - jj * PT, j = j_begin + jj;
        const int ax = a - ox, az = a - oz;
        TAP[jj * 2 * PT + a] = (ax >= 0 && ax < g.px) ? __ldg(fx + ((size_t)lp * ny + j) * g.px + ax) : 0.f;
        TAP[jj * 2 * PT + PT + a] = (az >= 0 && az < g.pz) ? __ldg(fz + ((size_t)lp * ny + j) * g.pz + az) : 0.f;
    }
    for (int e = tid; e < d.urows * d.apc; e += T) ACC[e] = 0.f;
    for (int e = tid; e < d.urows * d.kpu; e += T) U[e] = 0.f;  // zero k-halo columns (never written again)
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

// ============================================================================
// Fused transpose of the blur + attenuation, separable PSF.
//   V   nx rows x kpu: the detector plane, V[i][ZH + k], zero halo columns
//   Zb  nz rows x wp: k-adjoint of every V row, Zb[k][C + i], zero halo columns
//   MB  two plane buffers: each receives mubar(:, j, :) by TMA, is overwritten
//       in place with t = wbar * mubar, and leaves for the slab by a TMA bulk
//       store; the buffer of plane j+1 is loaded while plane j is computed.
// ============================================================================
template <int P, bool TILED>
__device__ __forceinline__ void adj_sep_body(const Geometry& g, const FusedDims& d, int cls_z,
                                             const float* __restrict__ vin, const float* __restrict__ mubar,
                                             const float* __restrict__ fx_adj, const float* __restrict__ fz_adj,
                                             float* __restrict__ slab, int l0, int* err, const int grp, const int v,
                                             const int tile)
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
    const int l = l0 + v;
    // output columns [i0, i0 + ti); their i-adjoint reads detector rows [vlo, vhi)
    // (untiled: the whole plane, with the constants folded at compile time)
    const int i0 = TILED ? (int)tile * d.TI : 0;
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

    // the first plane's attenuation is requested before anything else
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_load_1d(MB, mub + (size_t)j_begin * d.ps, SPECT_MBYTES, bar);
    }
    // the detector plane v(:,:,l), transposed, by asynchronous copies issued
    // next, so their latency overlaps the tap staging and the zeroing below
    for (int e = tid; e < nz * nvr; e += T) {
        const int k = e / nvr, r = e - k * nvr;
        cp_async_4(V + r * d.kpu + ZH + k, vin + (size_t)l * pln + (size_t)k * nx + vlo + r);
    }
    // edge-class taps of every plane of the group (zero-padded to P), also asynchronously
    for (int e = tid; e < (j_end - j_begin) * 3 * PT; e += T) {
        const int jj = e / (3 * PT), r3 = e - jj * 3 * PT, c = r3 / PT, a = r3 - c * PT, j = j_begin + jj;
        const int ax = a - ox, az = a - oz;
        const bool okx = ax >= 0 && ax < g.px, okz = c < cls_z && az >= 0 && az < g.pz;
        float* F = TAP + jj * 6 * PT;
        cp_async_4_or_zero(F + r3, okx ? fx_adj + ((size_t)c * nrow + (size_t)lp * ny + j) * g.px + ax : fx_adj, okx);
        cp_async_4_or_zero(F + 3 * PT + r3, okz ? fz_adj + ((size_t)c * nrow + (size_t)lp * ny + j) * g.pz + az : fz_adj,
                           okz);
    }

    // zero V outside the detector (the halo columns of the staged rows, and
    // whole rows beyond them) and Zb; then wait for the staged plane and taps
    const int halo = d.kpu - nz;  // zero columns of a staged row: [0, ZH) and [ZH + nz, kpu)
    for (int e = tid; e < nvr * halo; e += T) {
        const int r = e / halo, c = e - r * halo;
        V[r * d.kpu + (c < ZH ? c : c + nz)] = 0.f;
    }
    for (int e = nvr * d.kpu + tid; e < d.vrows * d.kpu; e += T) V[e] = 0.f;
    for (int e = tid; e < d.zarea; e += T) Zb[e] = 0.f;
    cp_async_wait_all();
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

// ---------------------------------------------------------------- host-side dimensioning
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
}  // namespace

}  // namespace spect
