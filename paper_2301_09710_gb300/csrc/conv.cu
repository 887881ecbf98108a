// conv.cu -- depth-dependent PSF blur and depth sum (Section II-A, Algorithm 1
// inner loop) and their transposes (Algorithm 2), in FP32 on the CUDA cores.
//
// Forward, for view l and depth plane j of the rotated, attenuated image w:
//   c_j(i,k) = sum_{a,b} p(a,b,j,l) w(clamp(i-a+cx), j, clamp(k-b+cz)),
//   v(i,k,l) = sum_j c_j(i,k)                               (replicate padding)
// Transpose, in gather form over the destination (i,k) of every plane j:
//   wbar_j(i,k) = sum_{a,b} p~(a,b) vext(i+a-cx, k+b-cz)
// with vext zero outside the detector and p~ = p for interior (i,k).  On the
// first/last row or column the replicate padding folds several taps onto one
// bin; there p~ is the matching edge-class variant of p: along an axis of
// length n >= 2, "low" (index 0) takes tail sums sum_{a>=a'} p(a) for
// a' >= c, "high" (index n-1) takes head sums sum_{a<=a'} p(a) for a' <= c;
// an axis of length 1 takes the full sum at the centre tap.  The variants are
// built once per plan (k_sep_variants / k_direct_variants_*).
//
// Accuracy: every per-depth blur is a short FP32 sum (<= px or pz terms per
// pass for the separable path, row partials for the direct path); the sum
// over depth uses Kahan compensation.
#include "spect_internal.cuh"

namespace spect {

namespace {
constexpr int kMaxOut = 16;    // outputs per thread, separable kernels
constexpr int kSepThreads = 256;
constexpr int kTI = 32, kTK = 32;  // direct kernels: output tile (i x k)
constexpr int kDirThreadsX = 32, kDirThreadsY = 8;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// edge class of index i on an axis of length n (slot in the variant arrays)
__device__ __forceinline__ int edge_class(int i, int n)
{
    if (n == 1) return 0;
    return i == 0 ? 1 : (i == n - 1 ? 2 : 0);
}
}  // namespace

// ============================================================================
// Forward, separable PSF p(a,b,j,l) = fx(a,j,l) fz(b,j,l).
// One block per (k-tile of Tk rows, view); the whole detector width per block,
// so the i-pass clamps inside shared memory and only the k-pass needs halo
// rows (Tk + 2cz staged rows, global row index clamped = replicate padding).
// ============================================================================
__global__ void __launch_bounds__(kSepThreads) k_conv_fwd_sep(Geometry g, const float* __restrict__ fx,
                                                              const float* __restrict__ fz,
                                                              const float* __restrict__ slab,
                                                              float* __restrict__ vout, int l0, int Tk,
                                                              const float* __restrict__ em_y,
                                                              const float* __restrict__ em_rbar)
{
    extern __shared__ float sm[];
    const int nx = g.nx, ny = g.ny, nz = g.nz, px = g.px, pz = g.pz;
    const int cx = (px - 1) / 2, cz = (pz - 1) / 2;
    const int R = Tk + 2 * cz;
    float* S = sm;             // R * nx
    float* Z = S + R * nx;     // Tk * nx
    float* FX = Z + Tk * nx;   // px
    float* FZ = FX + px;       // pz
    const int tid = threadIdx.x;
    const int v = blockIdx.y, l = l0 + v;
    const int k0 = blockIdx.x * Tk;
    const int tk = min(Tk, nz - k0);
    const int lp = g.nvp == 1 ? 0 : l;
    const int nout = tk * nx;
    const size_t nxy = (size_t)nx * ny;
    const float* base = slab + (size_t)v * nz * nxy;

    KSum acc[kMaxOut];
    for (int j = 0; j < ny; ++j) {
        for (int a = tid; a < px; a += kSepThreads) FX[a] = fx[((size_t)lp * ny + j) * px + a];
        for (int b = tid; b < pz; b += kSepThreads) FZ[b] = fz[((size_t)lp * ny + j) * pz + b];
        for (int e = tid; e < R * nx; e += kSepThreads) {
            const int r = e / nx, i = e - r * nx;
            const int gk = clampi(k0 - cz + r, 0, nz - 1);
            S[e] = base[(size_t)gk * nxy + (size_t)j * nx + i];
        }
        __syncthreads();
        // k-pass: Z(kk,i) = sum_b fz(b) w(clamp(k-b+cz), i)
        for (int e = tid; e < nout; e += kSepThreads) {
            const int kk = e / nx, i = e - kk * nx;
            const float* col = S + (kk + 2 * cz) * nx + i;
            float z = 0.f;
            for (int b = 0; b < pz; ++b) z = fmaf(FZ[b], col[-b * nx], z);
            Z[e] = z;
        }
        __syncthreads();
        // i-pass: c_j(kk,i) = sum_a fx(a) Z(kk, clamp(i-a+cx))
#pragma unroll
        for (int m = 0; m < kMaxOut; ++m) {
            const int e = tid + m * kSepThreads;
            if (e < nout) {
                const int kk = e / nx, i = e - kk * nx;
                const float* row = Z + kk * nx;
                float o = 0.f;
                for (int a = 0; a < px; ++a) o = fmaf(FX[a], row[clampi(i - a + cx, 0, nx - 1)], o);
                acc[m].add(o);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < kMaxOut; ++m) {
        const int e = tid + m * kSepThreads;
        if (e < nout) {
            const int kk = e / nx, i = e - kk * nx;
            const size_t o = ((size_t)l * nz + k0 + kk) * nx + i;
            const float val = acc[m].value();
            if (em_y) {
                const float yb = val + (em_rbar ? em_rbar[o] : 0.f);
                vout[o] = yb > 0.f ? em_y[o] / yb : 0.f;
            } else {
                vout[o] = val;
            }
        }
    }
}

// ============================================================================
// Forward, full (direct) PSF.  One block per (32x32 output tile, view); per
// depth plane the tile plus its halo (clamped = replicate padding) and the
// PSF plane are staged in shared memory; each thread owns 4 outputs.
// ============================================================================
__global__ void __launch_bounds__(kDirThreadsX* kDirThreadsY) k_conv_fwd_direct(
    Geometry g, const float* __restrict__ psf, const float* __restrict__ slab, float* __restrict__ vout, int l0,
    const float* __restrict__ em_y, const float* __restrict__ em_rbar)
{
    extern __shared__ float sm[];
    const int nx = g.nx, ny = g.ny, nz = g.nz, px = g.px, pz = g.pz;
    const int cx = (px - 1) / 2, cz = (pz - 1) / 2;
    const int WC = kTI + 2 * cx, WR = kTK + 2 * cz;
    float* W = sm;           // WR * WC
    float* P = W + WR * WC;  // pz * px
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kDirThreadsX + tx;
    const int nthr = kDirThreadsX * kDirThreadsY;
    const int i0 = blockIdx.x * kTI, k0 = blockIdx.y * kTK;
    const int v = blockIdx.z, l = l0 + v;
    const int lp = g.nvp == 1 ? 0 : l;
    const size_t nxy = (size_t)nx * ny;
    const float* base = slab + (size_t)v * nz * nxy;
    constexpr int M = kTK / kDirThreadsY;
    KSum acc[M];
    for (int j = 0; j < ny; ++j) {
        const float* pj = psf + ((size_t)lp * ny + j) * px * pz;
        for (int e = tid; e < px * pz; e += nthr) P[e] = pj[e];
        for (int e = tid; e < WR * WC; e += nthr) {
            const int r = e / WC, c = e - r * WC;
            const int gi = clampi(i0 - cx + c, 0, nx - 1), gk = clampi(k0 - cz + r, 0, nz - 1);
            W[e] = base[(size_t)gk * nxy + (size_t)j * nx + gi];
        }
        __syncthreads();
        float part[M];
#pragma unroll
        for (int m = 0; m < M; ++m) part[m] = 0.f;
        for (int b = 0; b < pz; ++b) {
            float rowp[M];
#pragma unroll
            for (int m = 0; m < M; ++m) rowp[m] = 0.f;
            const float* prow = P + b * px;
            for (int a = 0; a < px; ++a) {
                const float pv = prow[a];
#pragma unroll
                for (int m = 0; m < M; ++m)
                    rowp[m] = fmaf(pv, W[(ty + kDirThreadsY * m - b + 2 * cz) * WC + tx - a + 2 * cx], rowp[m]);
            }
#pragma unroll
            for (int m = 0; m < M; ++m) part[m] += rowp[m];
        }
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m].add(part[m]);
        __syncthreads();
    }
    const int i = i0 + tx;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int k = k0 + ty + kDirThreadsY * m;
        if (i < nx && k < nz) {
            const size_t o = ((size_t)l * nz + k) * nx + i;
            const float val = acc[m].value();
            if (em_y) {
                const float yb = val + (em_rbar ? em_rbar[o] : 0.f);
                vout[o] = yb > 0.f ? em_y[o] / yb : 0.f;
            } else {
                vout[o] = val;
            }
        }
    }
}

// ============================================================================
// Transpose, separable PSF.  One block per (k-tile, view).  The detector rows
// the tile needs (Tk + 2cz, zero outside the detector) are staged once; for
// every depth j (walked from the detector side so Eq. (1) is a running sum)
// the k-pass and i-pass adjoints with edge-class factors give wbar_j, which
// is multiplied by mubar and stored as t in slab[v][k][j][i].
// ============================================================================
__global__ void __launch_bounds__(kSepThreads) k_conv_adj_sep(Geometry g, int cls_z,
                                                              const float* __restrict__ fx_adj,
                                                              const float* __restrict__ fz_adj,
                                                              const ViewRot* __restrict__ rot,
                                                              const float* __restrict__ mu,
                                                              const float* __restrict__ vin,
                                                              float* __restrict__ slab, int l0, int Tk)
{
    extern __shared__ float sm[];
    const int nx = g.nx, ny = g.ny, nz = g.nz, px = g.px, pz = g.pz;
    const int cx = (px - 1) / 2, cz = (pz - 1) / 2;
    const int R = Tk + 2 * cz;
    float* V = sm;             // R * nx
    float* Z = V + R * nx;     // Tk * nx
    float* FX = Z + Tk * nx;   // 3 * px
    float* FZ = FX + 3 * px;   // cls_z * pz
    const int tid = threadIdx.x;
    const int v = blockIdx.y, l = l0 + v;
    const int k0 = blockIdx.x * Tk;
    const int tk = min(Tk, nz - k0);
    const int lp = g.nvp == 1 ? 0 : l;
    const int nout = tk * nx;
    const size_t nxy = (size_t)nx * ny;
    const size_t nrow = (size_t)g.nvp * ny;  // rows per class in the variant arrays
    const ViewRot r = rot[l];
    float* tbase = slab + (size_t)v * nz * nxy;

    for (int e = tid; e < R * nx; e += kSepThreads) {
        const int rr = e / nx, i = e - rr * nx;
        const int gk = k0 - cz + rr;
        V[e] = (gk >= 0 && gk < nz) ? vin[((size_t)l * nz + gk) * nx + i] : 0.f;
    }
    AttenScan sc[kMaxOut];
    for (int j = ny - 1; j >= 0; --j) {
        const size_t row = (size_t)lp * ny + j;
        for (int e = tid; e < 3 * px; e += kSepThreads) {
            const int c = e / px, a = e - c * px;
            FX[e] = fx_adj[((size_t)c * nrow + row) * px + a];
        }
        for (int e = tid; e < cls_z * pz; e += kSepThreads) {
            const int c = e / pz, b = e - c * pz;
            FZ[e] = fz_adj[((size_t)c * nrow + row) * pz + b];
        }
        __syncthreads();
        for (int e = tid; e < nout; e += kSepThreads) {
            const int kk = e / nx, i = e - kk * nx;
            const float* f = FZ + edge_class(k0 + kk, nz) * pz;
            const float* col = V + kk * nx + i;
            float z = 0.f;
            for (int b = 0; b < pz; ++b) z = fmaf(f[b], col[b * nx], z);
            Z[e] = z;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < kMaxOut; ++m) {
            const int e = tid + m * kSepThreads;
            if (e < nout) {
                const int kk = e / nx, i = e - kk * nx;
                const int k = k0 + kk;
                const float* f = FX + edge_class(i, nx) * px;
                const float* zr = Z + kk * nx;
                const int alo = max(0, cx - i), ahi = min(px, nx - i + cx);
                float wb = 0.f;
                for (int a = alo; a < ahi; ++a) wb = fmaf(f[a], zr[i + a - cx], wb);
                float mb = 1.f;
                if (g.has_mu) {
                    const Sample s = rot_sample(i, j, r, g.cint, g.cfrac);
                    mb = sc[m].step(gather_bilinear(mu + (size_t)k * nxy, s, nx, ny), g.dy);
                }
                tbase[(size_t)k * nxy + (size_t)j * nx + i] = wb * mb;
            }
        }
        __syncthreads();
    }
}

// ============================================================================
// Transpose, full PSF.  One block per (32x32 tile, view); the zero-extended
// detector tile with halo is staged once; per depth (from the detector side)
// interior outputs read the PSF plane from shared memory, edge outputs read
// their edge-class variant from global memory.
// ============================================================================
__global__ void __launch_bounds__(kDirThreadsX* kDirThreadsY) k_conv_adj_direct(
    Geometry g, int cls_z, const float* __restrict__ psf, const float* __restrict__ psf_adj,
    const ViewRot* __restrict__ rot, const float* __restrict__ mu, const float* __restrict__ vin,
    float* __restrict__ slab, int l0)
{
    extern __shared__ float sm[];
    const int nx = g.nx, ny = g.ny, nz = g.nz, px = g.px, pz = g.pz;
    const int cx = (px - 1) / 2, cz = (pz - 1) / 2;
    const int WC = kTI + 2 * cx, WR = kTK + 2 * cz;
    float* Vt = sm;           // WR * WC
    float* P = Vt + WR * WC;  // pz * px
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kDirThreadsX + tx;
    const int nthr = kDirThreadsX * kDirThreadsY;
    const int i0 = blockIdx.x * kTI, k0 = blockIdx.y * kTK;
    const int v = blockIdx.z, l = l0 + v;
    const int lp = g.nvp == 1 ? 0 : l;
    const size_t nxy = (size_t)nx * ny;
    const size_t pplane = (size_t)px * pz;
    const size_t nrow = (size_t)g.nvp * ny;
    const ViewRot r = rot[l];
    float* tbase = slab + (size_t)v * nz * nxy;
    constexpr int M = kTK / kDirThreadsY;

    for (int e = tid; e < WR * WC; e += nthr) {
        const int rr = e / WC, c = e - rr * WC;
        const int gi = i0 - cx + c, gk = k0 - cz + rr;
        Vt[e] = (gi >= 0 && gi < nx && gk >= 0 && gk < nz) ? vin[((size_t)l * nz + gk) * nx + gi] : 0.f;
    }
    const int i = i0 + tx;
    AttenScan sc[M];
    for (int j = ny - 1; j >= 0; --j) {
        const size_t row = (size_t)lp * ny + j;
        for (int e = tid; e < (int)pplane; e += nthr) P[e] = psf[row * pplane + e];
        __syncthreads();
        Sample s;
        if (g.has_mu) s = rot_sample(i, j, r, g.cint, g.cfrac);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int kk = ty + kDirThreadsY * m;
            const int k = k0 + kk;
            if (i < nx && k < nz) {
                const int ci = edge_class(i, nx), ck = edge_class(k, nz);
                float wb = 0.f;
                if (ci == 0 && ck == 0 && nz > 1) {
                    for (int b = 0; b < pz; ++b) {
                        const float* prow = P + b * px;
                        const float* vrow = Vt + (kk + b) * WC + tx;
                        float rp = 0.f;
                        for (int a = 0; a < px; ++a) rp = fmaf(prow[a], vrow[a], rp);
                        wb += rp;
                    }
                } else {
                    const float* pv = psf_adj + ((size_t)(ci * cls_z + ck) * nrow + row) * pplane;
                    for (int b = 0; b < pz; ++b) {
                        const float* vrow = Vt + (kk + b) * WC + tx;
                        float rp = 0.f;
                        for (int a = 0; a < px; ++a) rp = fmaf(__ldg(pv + b * px + a), vrow[a], rp);
                        wb += rp;
                    }
                }
                float mb = 1.f;
                if (g.has_mu) mb = sc[m].step(gather_bilinear(mu + (size_t)k * nxy, s, nx, ny), g.dy);
                tbase[(size_t)k * nxy + (size_t)j * nx + i] = wb * mb;
            }
        }
        __syncthreads();
    }
}

// ============================================================================
// Plan-time edge-class variants (FP64 sums, rounded once to FP32).
// ============================================================================
// sum of f(a) over the set of taps that edge class `cls` folds onto tap a'
__device__ double class_sum_1d(const float* f, int p, int cls, int n_axis, int ap, int stride)
{
    const int c = (p - 1) / 2;
    double s = 0.0;
    if (n_axis == 1) {  // both edges: every tap folds onto the centre
        if (ap == c)
            for (int a = 0; a < p; ++a) s += f[(size_t)a * stride];
        return s;
    }
    if (cls == 0) return f[(size_t)ap * stride];
    if (cls == 1) {
        if (ap >= c)
            for (int a = ap; a < p; ++a) s += f[(size_t)a * stride];
        return s;
    }
    if (ap <= c)
        for (int a = 0; a <= ap; ++a) s += f[(size_t)a * stride];
    return s;
}

__global__ void k_sep_variants(const float* __restrict__ f, float* __restrict__ out, int p, int nrows, int ncls,
                               int n_axis)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrows * p) return;
    const int row = idx / p, ap = idx - row * p;
    for (int c = 0; c < ncls; ++c)
        out[((size_t)c * nrows + row) * p + ap] = (float)class_sum_1d(f + (size_t)row * p, p, c, n_axis, ap, 1);
}

// stage 1: Q[ci][row][b][a'] = sum over the i-class set of a' of p(a,b)
__global__ void k_direct_variants_a(const float* __restrict__ psf, float* __restrict__ Q, int px, int pz, int nrows,
                                    int ncls_x, int nx)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t plane = (size_t)px * pz;
    if (idx >= (size_t)nrows * plane) return;
    const size_t row = idx / plane;
    const int e = (int)(idx - row * plane), b = e / px, ap = e - b * px;
    const float* pr = psf + row * plane + (size_t)b * px;
    for (int c = 0; c < ncls_x; ++c)
        Q[((size_t)c * nrows + row) * plane + e] = (float)class_sum_1d(pr, px, c, nx, ap, 1);
}

// stage 2: out[ci*cls_z+ck][row][b'][a'] = sum over the k-class set of b' of Q[ci][row][b][a']
__global__ void k_direct_variants_b(const float* __restrict__ Q, float* __restrict__ out, int px, int pz, int nrows,
                                    int ncls_x, int ncls_z, int nz)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t plane = (size_t)px * pz;
    if (idx >= (size_t)nrows * plane) return;
    const size_t row = idx / plane;
    const int e = (int)(idx - row * plane), bp = e / px, ap = e - bp * px;
    for (int ci = 0; ci < ncls_x; ++ci) {
        const float* qc = Q + ((size_t)ci * nrows + row) * plane + ap;
        for (int ck = 0; ck < ncls_z; ++ck)
            out[((size_t)(ci * ncls_z + ck) * nrows + row) * plane + e] =
                (float)class_sum_1d(qc, pz, ck, nz, bp, px);
    }
}

// ============================================================================
// launchers
// ============================================================================
static size_t sep_smem_bytes(const Geometry& g, int Tk, bool adjoint, int cls_z)
{
    const int R = Tk + 2 * ((g.pz - 1) / 2);
    size_t n = (size_t)R * g.nx + (size_t)Tk * g.nx;
    n += adjoint ? (size_t)3 * g.px + (size_t)cls_z * g.pz : (size_t)g.px + g.pz;
    return n * sizeof(float);
}

static size_t direct_smem_bytes(const Geometry& g)
{
    const size_t WC = kTI + 2 * ((g.px - 1) / 2), WR = kTK + 2 * ((g.pz - 1) / 2);
    return (WR * WC + (size_t)g.px * g.pz) * sizeof(float);
}

// Largest k-tile that fits shared memory and the per-thread output budget.
int choose_sep_tile(const Geometry& g, int cls_z, size_t smem_limit)
{
    int Tk = kMaxOut * kSepThreads / g.nx;
    Tk = min(Tk, g.nz);
    while (Tk > 1 && (sep_smem_bytes(g, Tk, true, cls_z) > smem_limit || sep_smem_bytes(g, Tk, false, cls_z) > smem_limit))
        --Tk;
    if (Tk < 1 || sep_smem_bytes(g, Tk, true, cls_z) > smem_limit) return 0;
    // prefer enough blocks to fill the GPU: shrink while a view has < 4 tiles
    while (Tk > 8 && (g.nz + Tk - 1) / Tk < 4) Tk = (Tk + 1) / 2;
    return Tk;
}

bool direct_fits(const Geometry& g, size_t smem_limit) { return direct_smem_bytes(g) <= smem_limit; }

cudaError_t launch_conv_forward(const spect_plan_s& P, float* v, int l0, int nv, const float* em_y,
                                const float* em_rbar, cudaStream_t st)
{
    const Geometry& g = P.g;
    if (P.separable) {
        const int Tk = P.sep_tk;
        const size_t smem = sep_smem_bytes(g, Tk, false, P.cls_z);
        cudaFuncSetAttribute(k_conv_fwd_sep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid((g.nz + Tk - 1) / Tk, nv);
        k_conv_fwd_sep<<<grid, kSepThreads, smem, st>>>(g, P.fx, P.fz, P.slab, v, l0, Tk, em_y, em_rbar);
    } else {
        const size_t smem = direct_smem_bytes(g);
        cudaFuncSetAttribute(k_conv_fwd_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid((g.nx + kTI - 1) / kTI, (g.nz + kTK - 1) / kTK, nv);
        k_conv_fwd_direct<<<grid, dim3(kDirThreadsX, kDirThreadsY), smem, st>>>(g, P.psf, P.slab, v, l0, em_y,
                                                                                em_rbar);
    }
    return cudaGetLastError();
}

cudaError_t launch_conv_adjoint(const spect_plan_s& P, const float* v, int l0, int nv, cudaStream_t st)
{
    const Geometry& g = P.g;
    if (P.separable) {
        const int Tk = P.sep_tk;
        const size_t smem = sep_smem_bytes(g, Tk, true, P.cls_z);
        cudaFuncSetAttribute(k_conv_adj_sep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid((g.nz + Tk - 1) / Tk, nv);
        k_conv_adj_sep<<<grid, kSepThreads, smem, st>>>(g, P.cls_z, P.fx_adj, P.fz_adj, P.rot, P.mu, v, P.slab, l0,
                                                        Tk);
    } else {
        const size_t smem = direct_smem_bytes(g);
        cudaFuncSetAttribute(k_conv_adj_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid((g.nx + kTI - 1) / kTI, (g.nz + kTK - 1) / kTK, nv);
        k_conv_adj_direct<<<grid, dim3(kDirThreadsX, kDirThreadsY), smem, st>>>(g, P.cls_z, P.psf, P.psf_adj,
                                                                                P.rot, P.mu, v, P.slab, l0);
    }
    return cudaGetLastError();
}

cudaError_t launch_psf_variants(spect_plan_s& P, float* scratch, cudaStream_t st)
{
    const Geometry& g = P.g;
    const int nrows = g.nvp * g.ny;
    if (P.separable) {
        k_sep_variants<<<(nrows * g.px + 255) / 256, 256, 0, st>>>(P.fx, P.fx_adj, g.px, nrows, 3, g.nx);
        k_sep_variants<<<(nrows * g.pz + 255) / 256, 256, 0, st>>>(P.fz, P.fz_adj, g.pz, nrows, P.cls_z, g.nz);
    } else {
        const size_t n = (size_t)nrows * g.px * g.pz;
        const unsigned blocks = (unsigned)((n + 255) / 256);
        k_direct_variants_a<<<blocks, 256, 0, st>>>(P.psf, scratch, g.px, g.pz, nrows, P.cls_x, g.nx);
        k_direct_variants_b<<<blocks, 256, 0, st>>>(scratch, P.psf_adj, g.px, g.pz, nrows, P.cls_x, P.cls_z, g.nz);
    }
    return cudaGetLastError();
}

}  // namespace spect
