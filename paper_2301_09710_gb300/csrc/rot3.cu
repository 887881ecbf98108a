// rot3.cu -- the three-pass image rotation of the projector on the fused path.
//
// Section II-A of arXiv 2301.09710 implements two image rotations: bilinear
// interpolation (the default here) and 3-pass 1D linear interpolation, both
// with zero padding.  The three-pass rotation by theta:
//   theta = q*pi/2 + phi, q the nearest integer, phi in [-pi/4, pi/4];
//   the exact quarter turn q (the bilinear convention at theta = q*pi/2),
//   then three pull-backs, each a 1D linear interpolation with zero padding:
//     pass 1 along x at i + tan(phi/2)(j-c),
//     pass 2 along y at j - sin(phi)(i-c),
//     pass 3 along x at i + tan(phi/2)(j-c),
//   whose product samples at R(-phi)(p-c)+c, the convention of the bilinear
//   rotation (content turns by +theta about c = (nx-1)/2).
//
// Every pass reads two neighbours along one axis, so two passes read four:
//   A:  passes 1 (with the quarter turn) and 2 together are one 4-tap gather
//       (k_gather4) from x_t into a per-view [j][i][k] volume; pass 3 runs as
//       the fused rotation kernel (k_rot_fwd, fused.cu) on that volume with a
//       table in the bilinear format (four slot weights, one base pixel), so
//       attenuation and the blur kernel's plane images are unchanged.
//   A': the transpose of pass 3 is a 2-tap gather in the same table format
//       (k_table_gather; the transpose of a 1D linear shift by d is the shift
//       by -d with the same weights); the transposes of passes 2 and 1, of
//       the quarter turn and the sum over views run as the list gather
//       (k_adj_rot_t), whose fixed-length lists hold the four entries of every
//       (voxel, view).
//   The attenuation cache of Eq. (1) is built from mu turned the same way.
// Offsets and weights are computed in FP64 on the host and rounded once to
// FP32 (a two-pass weight is the FP64 product rounded); the forward taps and
// the adjoint entries use the same FP32 weights.
#include <cmath>
#include <cstring>
#include <vector>

#include "spect_internal.cuh"

namespace spect {

namespace {

struct Rot3View {
    int q;     // quarter turns
    double t;  // tan(phi / 2)
    double s;  // sin(phi)
};

Rot3View rot3_view(double theta)
{
    const double r = std::nearbyint(theta / (M_PI / 2.0));
    const double phi = theta - r * (M_PI / 2.0);
    Rot3View v;
    v.q = (int)(((long)r % 4 + 4) % 4);
    v.t = std::tan(0.5 * phi);
    v.s = std::sin(phi);
    return v;
}

// A row or column shift d = o + a (o integer, 0 <= a < 1): the output at
// position u reads the input at u + o (weight 1 - a) and u + o + 1 (weight a).
struct Shift {
    int o;
    double w[2];  // 1 - a, a
};

Shift make_shift(double d)
{
    const double f = std::floor(d);
    const double a = d - f;
    Shift s;
    s.o = (int)f;
    s.w[0] = 1.0 - a;
    s.w[1] = a;
    return s;
}

// Pixel of the unrotated frame that the quarter turn q brings to (i, j).
void quarter_from(int n, int q, int i, int j, int* si, int* sj)
{
    switch (q) {
        case 0: *si = i; *sj = j; break;
        case 1: *si = j; *sj = n - 1 - i; break;
        case 2: *si = n - 1 - i; *sj = n - 1 - j; break;
        default: *si = n - 1 - j; *sj = i; break;
    }
}

// The pixel (i, j) of the turned frame that the quarter turn q fills from (si, sj).
void quarter_to(int n, int q, int si, int sj, int* i, int* j)
{
    switch (q) {
        case 0: *i = si; *j = sj; break;
        case 1: *i = n - 1 - sj; *j = si; break;
        case 2: *i = n - 1 - si; *j = n - 1 - sj; break;
        default: *i = sj; *j = n - 1 - si; break;
    }
}

// Table entry (slot weights, base pixel) of an output reading up to two
// pixels of an n x n frame; pixels outside the frame are dropped (zero
// padding).  Slots (0,0), (1,0), (0,1), (1,1) are relative to the base,
// which is clamped so all four stay inside the frame.
void put_entry(int n, const int (&pi)[2], const int (&pj)[2], const float (&w)[2], float* wout, int* base)
{
    int mi = n, mj = n;
    bool any = false;
    for (int m = 0; m < 2; ++m)
        if (pi[m] >= 0 && pi[m] < n && pj[m] >= 0 && pj[m] < n) {
            mi = std::min(mi, pi[m]);
            mj = std::min(mj, pj[m]);
            any = true;
        }
    for (int s = 0; s < 4; ++s) wout[s] = 0.f;
    *base = 0;
    if (!any) return;
    const int bi = std::min(std::max(mi, 0), n - 2), bj = std::min(std::max(mj, 0), n - 2);
    for (int m = 0; m < 2; ++m)
        if (pi[m] >= 0 && pi[m] < n && pj[m] >= 0 && pj[m] < n) wout[(pi[m] - bi) + 2 * (pj[m] - bj)] += w[m];
    *base = bi + n * bj;
}

}  // namespace

// ============================================================================
// Device kernels
// ============================================================================

// out[v] (plane stride out_ps, view stride out_vs) at (j, i, k) = the four
// slots of table entry (l0 + v, j, i) applied to in[v] (plane stride in_ps,
// view stride in_vs; in_vs = 0: every view reads the same volume).
// One block per (row j, view); threads over (i, k) with k fastest, so the
// slot reads are coalesced runs along k.
__global__ void __launch_bounds__(256) k_table_gather(Geometry g, int ts, const float* __restrict__ tab,
                                                      const float* __restrict__ in, size_t in_vs, int in_ps,
                                                      float* __restrict__ out, size_t out_vs, int out_ps, int l0)
{
    const int j = blockIdx.x, v = blockIdx.y, l = l0 + v;
    const float* blk = tab + ((size_t)l * g.ny + j) * ts;
    const float4* TW = reinterpret_cast<const float4*>(blk);
    const int* TB = reinterpret_cast<const int*>(blk + 4 * g.nx);
    const float* src = in + (size_t)v * in_vs;
    float* dst = out + (size_t)v * out_vs + (size_t)j * out_ps;
    const int n = g.nx * g.nz;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / g.nz, k = e - i * g.nz;
        const float4 w = __ldg(TW + i);
        const int b = __ldg(TB + i);
        const int bj = b / g.nx, bi = b - bj * g.nx;
        const float* p = src + (size_t)bj * in_ps + (size_t)bi * g.nz + k;
        float acc = w.x * __ldg(p);
        acc = fmaf(w.y, __ldg(p + g.nz), acc);
        acc = fmaf(w.z, __ldg(p + in_ps), acc);
        acc = fmaf(w.w, __ldg(p + in_ps + g.nz), acc);
        dst[(size_t)i * g.nz + k] = acc;
    }
}

// out[v] (plane stride out_ps, view stride out_vs) at (j, i, k) =
// sum_m w_m in[k + off_m] for the four (weight, element offset) taps of entry
// (l0 + v, j, i): per (l, j) block, nx float4 weights then nx int4 offsets
// into one [j][i][k] input volume (taps outside the frame have weight 0 and
// offset 0).  Threads over (i, k), k fastest: coalesced runs along k.
__global__ void __launch_bounds__(256) k_gather4(Geometry g, int ts4, const float* __restrict__ tab,
                                                 const float* __restrict__ in, float* __restrict__ out,
                                                 size_t out_vs, int out_ps, int l0)
{
    const int j = blockIdx.x, v = blockIdx.y, l = l0 + v;
    const float* blk = tab + ((size_t)l * g.ny + j) * ts4;
    const float4* TW = reinterpret_cast<const float4*>(blk);
    const int4* TO = reinterpret_cast<const int4*>(blk + 4 * g.nx);
    float* dst = out + (size_t)v * out_vs + (size_t)j * out_ps;
    const int n = g.nx * g.nz;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / g.nz, k = e - i * g.nz;
        const float4 w = __ldg(TW + i);
        const int4 o = __ldg(TO + i);
        const float* p = in + k;
        float acc = w.x * __ldg(p + o.x);
        acc = fmaf(w.y, __ldg(p + o.y), acc);
        acc = fmaf(w.z, __ldg(p + o.z), acc);
        acc = fmaf(w.w, __ldg(p + o.w), acc);
        dst[(size_t)i * g.nz + k] = acc;
    }
}

// mubar[l][j][i][k] from the rotated map mu~ of view l ([j][i][k], dense):
// Eq. (1) walked from the detector side, as k_mubar_cache does for the
// bilinear rotation.
__global__ void k_mubar_rotated(Geometry g, int ps, const float* __restrict__ mu_rot, int l,
                                float* __restrict__ mubar)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int per = g.nx * g.nz;
    if (idx >= per) return;
    const size_t pln = (size_t)per;
    AttenScan sc;
    for (int j = g.ny - 1; j >= 0; --j) {
        const float m = mu_rot[(size_t)j * pln + idx];
        mubar[((size_t)l * g.ny + j) * ps + idx] = g.has_mu ? sc.step(m, g.dy) : 1.f;
    }
}

// ============================================================================
// Host: tables, lists and the attenuation cache
// ============================================================================


// Floats per (view, row) block of the two-pass table: nx float4 weights, nx int4 offsets.
int rot3_ts4(int nx) { return 8 * nx; }

cudaError_t build_rot3(spect_plan_s& P, const double* angles, const float* mu_t, cudaStream_t st)
{
    const Geometry& g = P.g;
    const int n = g.nx, nz = g.nz, nview = g.nview, ts = P.ts, ts4 = rot3_ts4(n), ps = P.ps, E = P.adj_max;
    if (E < 4) return cudaErrorInvalidValue;  // the lists hold four entries per (voxel, view)
    const double c = 0.5 * (double)(n - 1);
    const size_t pln = (size_t)n * nz, nxy = (size_t)n * n, vol = nxy * nz;
    const size_t blk = (size_t)nview * n * ts, blk4 = (size_t)nview * n * ts4;
    std::vector<float> tp12(blk4, 0.f), tp3(blk, 0.f), tt3(blk, 0.f);
    std::vector<AdjEntry> lists(nxy * nview * (size_t)E);
    std::vector<Shift> rows(n), cols(n);
    for (int l = 0; l < nview; ++l) {
        const double th = angles ? angles[l] : 2.0 * M_PI * (double)l / (double)nview;
        const Rot3View rv = rot3_view(th);
        for (int m = 0; m < n; ++m) {
            rows[m] = make_shift(rv.t * ((double)m - c));   // passes 1 and 3, row m
            cols[m] = make_shift(-rv.s * ((double)m - c));  // pass 2, column m
        }
        for (int j = 0; j < n; ++j) {
            float* w12 = &tp12[((size_t)l * n + j) * ts4];
            int* o12 = reinterpret_cast<int*>(w12 + 4 * n);
            float* w3 = &tp3[((size_t)l * n + j) * ts];
            float* w3t = &tt3[((size_t)l * n + j) * ts];
            int* b3 = reinterpret_cast<int*>(w3 + 4 * n);
            int* b3t = reinterpret_cast<int*>(w3t + 4 * n);
            const Shift& r = rows[j];
            const float rw[2] = {(float)r.w[0], (float)r.w[1]};
            for (int i = 0; i < n; ++i) {
                // passes 1 + 2: column i at rows j + o_i + m' (pass 2), each row r at
                // quarter-turned columns i + o_r + m (pass 1); weight w_m'(i) w_m(r)
                int cnt = 0;
                const Shift& cs = cols[i];
                for (int mp = 0; mp < 2; ++mp) {
                    const int rr = j + cs.o + mp;
                    if (rr < 0 || rr >= n) continue;
                    const Shift& r1 = rows[rr];
                    for (int m = 0; m < 2; ++m) {
                        const int hi = i + r1.o + m;
                        if (hi < 0 || hi >= n) continue;
                        int si, sj;
                        quarter_from(n, rv.q, hi, rr, &si, &sj);
                        w12[4 * i + cnt] = (float)(cs.w[mp] * r1.w[m]);
                        o12[4 * i + cnt] = sj * (int)pln + si * nz;
                        ++cnt;
                    }
                }
                for (; cnt < 4; ++cnt) {
                    w12[4 * i + cnt] = 0.f;
                    o12[4 * i + cnt] = 0;
                }
                // pass 3: row j at (i + o, j), (i + o + 1, j)
                {
                    const int pi[2] = {i + r.o, i + r.o + 1}, pj[2] = {j, j};
                    put_entry(n, pi, pj, rw, w3 + 4 * i, b3 + i);
                }
                // pass 3 transposed: row j at (i - o, j) with w0, (i - o - 1, j) with w1
                {
                    const int pi[2] = {i - r.o, i - r.o - 1}, pj[2] = {j, j};
                    put_entry(n, pi, pj, rw, w3t + 4 * i, b3t + i);
                }
            }
        }
        // passes 1 and 2 transposed and the quarter turn transposed: voxel column q
        // receives, from view l, the pass-2 inputs that reach it (four at most)
        for (int qj = 0; qj < n; ++qj)
            for (int qi = 0; qi < n; ++qi) {
                int hi, hj;
                quarter_to(n, rv.q, qi, qj, &hi, &hj);
                const Shift& r = rows[hj];
                AdjEntry* e = &lists[(((size_t)qi + (size_t)n * qj) * nview + l) * E];
                int cnt = 0;
                for (int m = 0; m < 2; ++m) {
                    const int c1 = hi - r.o - m;  // pass-1 output column that read (hi, hj)
                    if (c1 < 0 || c1 >= n) continue;
                    const Shift& cs = cols[c1];
                    for (int mp = 0; mp < 2; ++mp) {
                        const int rr = hj - cs.o - mp;  // pass-2 output row that read (c1, hj)
                        const float w = (float)(cs.w[mp] * r.w[m]);
                        if (rr < 0 || rr >= n || w == 0.f) continue;
                        e[cnt].p = rr * ps + c1 * nz;  // [j][i][k] volume with plane stride ps
                        e[cnt].w = w;
                        ++cnt;
                    }
                }
                for (; cnt < E; ++cnt) {
                    e[cnt].p = 0;
                    e[cnt].w = 0.f;
                }
            }
    }
    cudaError_t e = cudaMemcpyAsync(P.r3_p12, tp12.data(), blk4 * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.rtab, tp3.data(), blk * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.r3_t3, tt3.data(), blk * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.adjf, lists.data(), lists.size() * sizeof(AdjEntry), cudaMemcpyHostToDevice, st);
    // the attenuation cache from mu turned by the same passes, view by view
    for (int l = 0; l < nview && e == cudaSuccess; ++l) {
        const dim3 grid(n, 1);
        k_gather4<<<grid, 256, 0, st>>>(g, ts4, P.r3_p12, mu_t, P.r3_a, vol, (int)pln, l);
        k_table_gather<<<grid, 256, 0, st>>>(g, ts, P.rtab, P.r3_a, vol, (int)pln, P.r3_b, vol, (int)pln, l);
        k_mubar_rotated<<<(unsigned)((pln + 255) / 256), 256, 0, st>>>(g, ps, P.r3_b, l, P.mubar);
        e = cudaGetLastError();
    }
    // the host vectors must outlive the asynchronous uploads
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

// A: passes 1 and 2 of views [l0, l0 + nv) from x_t into r3_b (dense [j][i][k] per view).
cudaError_t launch_rot3_forward_passes(const spect_plan_s& P, const float* xt, int l0, int nv, cudaStream_t st)
{
    const Geometry& g = P.g;
    const size_t pln = (size_t)g.nx * g.nz;
    k_gather4<<<dim3(g.ny, nv), 256, 0, st>>>(g, rot3_ts4(g.nx), P.r3_p12, xt, P.r3_b, pln * g.ny, (int)pln, l0);
    return cudaGetLastError();
}

// A': pass 3 transposed, views [l0, l0 + nv): the t planes of the work slab
// (plane stride ps) into r3_a (plane stride ps), which the list gather reads.
cudaError_t launch_rot3_adjoint_passes(const spect_plan_s& P, int l0, int nv, cudaStream_t st)
{
    const Geometry& g = P.g;
    const size_t vs = (size_t)g.ny * P.ps;
    k_table_gather<<<dim3(g.ny, nv), 256, 0, st>>>(g, P.ts, P.r3_t3, P.slab, vs, P.ps, P.r3_a, vs, P.ps, l0);
    return cudaGetLastError();
}

}  // namespace spect
