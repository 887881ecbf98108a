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
// Every pass reads two neighbours along one axis, so the three passes read
// eight pixels of the quarter-turned frame, with weights that are products of
// the three passes' linear-interpolation weights:
//   A:  the fused rotation kernel's eight-tap variant (k_rot_fwd8, fused.cu)
//       gathers them from x_t per output (view, row, column), attenuates and
//       writes the blur kernel's plane images -- no pass volumes in between.
//   A': the transposes of passes 3, 2 and 1, of the quarter turn and the sum
//       over views run as the adjacency-list gather (patch or list form), whose
//       fixed-length lists hold the eight entries of every (voxel, view) and
//       read the t planes the adjoint blur writes, as for bilinear rotation.
//   The attenuation cache of Eq. (1) is built at plan time from mu turned
//   by the same eight-tap table.
// Offsets and weights are computed in FP64 on the host; each tap weight is
// the FP64 product of its three pass weights, rounded once to FP32, and the
// forward taps and the adjoint entries use the same FP32 weights.
#include <cmath>
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

}  // namespace

// ============================================================================
// Device kernels
// ============================================================================

// out (dense [j][i][k]) at (j, i, k) = sum_m w_m in[k + off_m] over the N
// (weight, element offset) taps of entry (l, j, i) of a table whose (l, j)
// block holds nx groups of N weights then nx groups of N int offsets into one
// [j][i][k] volume (unused taps: weight 0, offset 0).  Plan time only (the
// attenuation cache); the projector itself runs the taps in k_rot_fwd8.
template <int N>
__global__ void __launch_bounds__(256) k_gather_taps(Geometry g, int tsn, const float* __restrict__ tab,
                                                     const float* __restrict__ in, float* __restrict__ out, int l)
{
    const int j = blockIdx.x;
    const float* blk = tab + ((size_t)l * g.ny + j) * tsn;
    const int* off = reinterpret_cast<const int*>(blk + N * g.nx);
    float* dst = out + (size_t)j * g.nx * g.nz;
    const int n = g.nx * g.nz;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / g.nz, k = e - i * g.nz;
        const float* w = blk + N * i;
        const int* o = off + N * i;
        float acc = w[0] * __ldg(in + o[0] + k);
#pragma unroll
        for (int m = 1; m < N; ++m) acc = fmaf(w[m], __ldg(in + o[m] + k), acc);
        dst[(size_t)i * g.nz + k] = acc;
    }
}

// mubar[l][j][i][k] from the rotated map mu~ of view l ([j][i][k], dense):
// Eq. (1) walked from the detector side with a compensated running sum, one
// thread per (i, k) column (coalesced), the same arithmetic as the bilinear
// rotation's attenuation cache (k_mubar_cache).
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
// Host: the eight-tap table, the eight-entry lists, the attenuation cache
// ============================================================================

int rot3_ts8(int nx) { return 16 * nx; }

cudaError_t build_rot3(spect_plan_s& P, const double* angles, const float* mu_t, float* scratch, cudaStream_t st)
{
    const Geometry& g = P.g;
    const int n = g.nx, nz = g.nz, nview = g.nview, ts8 = rot3_ts8(n), ps = P.ps, E = P.adj_max;
    if (E < 8) return cudaErrorInvalidValue;  // the lists hold eight entries per (voxel, view)
    const double c = 0.5 * (double)(n - 1);
    const size_t pln = (size_t)n * nz, nxy = (size_t)n * n;
    std::vector<float> tab((size_t)nview * n * ts8, 0.f);
    std::vector<AdjEntry> lists(nxy * nview * (size_t)E);
    std::vector<Shift> rows(n), cols(n);
    for (int l = 0; l < nview; ++l) {
        const double th = angles ? angles[l] : 2.0 * M_PI * (double)l / (double)nview;
        const Rot3View rv = rot3_view(th);
        for (int m = 0; m < n; ++m) {
            rows[m] = make_shift(rv.t * ((double)m - c));   // passes 1 and 3, row m
            cols[m] = make_shift(-rv.s * ((double)m - c));  // pass 2, column m
        }
        // A: output (i, j) <- pass 3 at (i + o_j + m3, j) <- pass 2 at (i2, j + o_i2 + mp)
        //    <- pass 1 at quarter-turned (i2 + o_r + m, r)
        for (int j = 0; j < n; ++j) {
            float* w = &tab[((size_t)l * n + j) * ts8];
            int* o = reinterpret_cast<int*>(w + 8 * n);
            for (int i = 0; i < n; ++i) {
                int cnt = 0;
                for (int m3 = 0; m3 < 2; ++m3) {
                    const int i2 = i + rows[j].o + m3;
                    if (i2 < 0 || i2 >= n) continue;
                    const Shift& cs = cols[i2];
                    for (int mp = 0; mp < 2; ++mp) {
                        const int r = j + cs.o + mp;
                        if (r < 0 || r >= n) continue;
                        for (int m = 0; m < 2; ++m) {
                            const int hi = i2 + rows[r].o + m;
                            if (hi < 0 || hi >= n) continue;
                            int si, sj;
                            quarter_from(n, rv.q, hi, r, &si, &sj);
                            w[8 * i + cnt] = (float)((cs.w[mp] * rows[r].w[m]) * rows[j].w[m3]);
                            o[8 * i + cnt] = sj * (int)pln + si * nz;
                            ++cnt;
                        }
                    }
                }
                for (; cnt < 8; ++cnt) {
                    w[8 * i + cnt] = 0.f;
                    o[8 * i + cnt] = 0;
                }
            }
        }
        // A': voxel column q receives from view l the t-plane pixels whose taps read
        // it -- passes 1, 2, 3 transposed after the quarter turn transposed
        for (int qj = 0; qj < n; ++qj)
            for (int qi = 0; qi < n; ++qi) {
                int hi, hj;
                quarter_to(n, rv.q, qi, qj, &hi, &hj);
                AdjEntry* e = &lists[(((size_t)qi + (size_t)n * qj) * nview + l) * E];
                int cnt = 0;
                for (int m = 0; m < 2; ++m) {
                    const int c1 = hi - rows[hj].o - m;  // pass-1 output column that read (hi, hj)
                    if (c1 < 0 || c1 >= n) continue;
                    const Shift& cs = cols[c1];
                    for (int mp = 0; mp < 2; ++mp) {
                        const int r = hj - cs.o - mp;  // pass-2 output row that read (c1, hj)
                        if (r < 0 || r >= n) continue;
                        for (int m3 = 0; m3 < 2; ++m3) {
                            const int c3 = c1 - rows[r].o - m3;  // pass-3 output column that read (c1, r)
                            const float wt = (float)((cs.w[mp] * rows[hj].w[m]) * rows[r].w[m3]);
                            if (c3 < 0 || c3 >= n || wt == 0.f) continue;
                            e[cnt].p = r * ps + c3 * nz;  // the t plane r, column c3 (plane stride ps)
                            e[cnt].w = wt;
                            ++cnt;
                        }
                    }
                }
                for (; cnt < E; ++cnt) {
                    e[cnt].p = 0;
                    e[cnt].w = 0.f;
                }
            }
    }
    cudaError_t e = cudaMemcpyAsync(P.r3_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.adjf, lists.data(), lists.size() * sizeof(AdjEntry), cudaMemcpyHostToDevice, st);
    // the attenuation cache from mu turned by the same taps, view by view
    for (int l = 0; l < nview && e == cudaSuccess; ++l) {
        k_gather_taps<8><<<n, 256, 0, st>>>(g, ts8, P.r3_tab, mu_t, scratch, l);
        k_mubar_rotated<<<(unsigned)((pln + 255) / 256), 256, 0, st>>>(g, ps, scratch, l, P.mubar);
        e = cudaGetLastError();
    }
    // the host vectors must outlive the asynchronous uploads
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

}  // namespace spect
